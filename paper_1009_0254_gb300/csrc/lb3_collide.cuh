// lb3_collide.cuh -- the per-node fluctuating collision on the D3Q19 lattice.
//
// [GACV] Sec. IV states that the lattice fluctuation-dissipation derivation of the noise
// holds on any DdQn lattice; this is the paper's D2Q9 model carried to D3Q19:
//   basis   the weighted-orthogonal modes of Duenweg, Schiller & Ladd, Phys. Rev. E 76,
//           036704 (2007), Table I: rho, j, bulk c^2 - 1, five shear modes, nine ghosts
//   m^eq    rho, j, the trace and traceless part of P^th + rho u u (Eq. press-ten with
//           p0 = cs2 rho, or the double well's bulk pressure, Coef3); the isotropic
//           fourth-order ghost e16 = -3 (p0 - rho/3 - kappa rho lap rho) - (9/2) kappa |grad rho|^2 (the
//           choice that reduces to Table II on fields uniform along an axis); other ghosts 0
//   relax   m*_a = m_a + lambda_a (m_a - m_a^eq) + xi_a (Eq. fluct-lin-lbe)
//   noise   xi = L nu with L L^T = Xi(0) (Eq. noise-matrix-k0), two Philox draws per node
//   back    f*_i = f_i + w_i sum_a T_ai (m*_a - m_a) / N_a.
// Everything is on deviations from the rest state fbar_i in the arithmetic type R.
//
// Velocity order (the ABI's): 0 rest; 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z; the edges
// 7 (1,1,0), 8 (1,-1,0), 9 (-1,1,0), 10 (-1,-1,0), 11 (0,1,1), 12 (0,1,-1), 13 (0,-1,1),
// 14 (0,-1,-1), 15 (1,0,1), 16 (-1,0,1), 17 (1,0,-1), 18 (-1,0,-1).  Opposite pairs:
// A = (7,10) along (1,1,0), B = (8,9) along (1,-1,0), C = (11,14) along (0,1,1),
// D = (12,13) along (0,1,-1), E = (15,18) along (1,0,1), F = (16,17) along (-1,0,1).
#pragma once

#include <cstdint>

namespace lbf3 {

constexpr int Q3 = 19;

// Density deviations at the node (c) and at its 18 neighbours r + c_i: faces xp = +x ...,
// edges ap = r + (1,1,0), am = r - (1,1,0), and so on for the pairs B..F.
template <typename R>
struct Rho3 {
    R c, xp, xm, yp, ym, zp, zm;
    R ap, am, bp, bm, cp, cm, dp, dm, ep, em, fp, fm;
};

// Coefficients of one run in the arithmetic type.  The bulk pressure relative to the rest
// state is p0(rho0 + dr) - p0(rho0) = dr (cs2 + dr (e2 + dr (e3 + dr e4))): e2..e4 are zero
// for p0 = cs2 rho and the double well's quartic otherwise (Sec. II A).
template <typename R>
struct Coef3 {
    R rho0, d, kappa;          // d = 3 cs2 - 1: weight of the pressure deviation in e4, e16
    R lb, ls, lg;              // lambda of the bulk, shear and ghost modes
    R e2, e3, e4;              // higher coefficients of the bulk pressure
};

// 3 (p0(rho0 + dr) - p0(rho0)) - dr = dd dr: the slope of the pressure deviation in the
// trace and ghost equilibria (exactly d when e2..e4 are zero)
template <typename R>
__host__ __device__ __forceinline__ R pressure_slope(const Coef3<R>& a, R dr) {
    return a.d + R(3) * dr * (a.e2 + dr * (a.e3 + dr * a.e4));
}

// 1/x: the hardware approximation in FP32 device code (relative error below 2^-22), IEEE
// division otherwise
__host__ __device__ __forceinline__ float recip19(float x) {
#ifdef __CUDA_ARCH__
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#else
    return 1.0f / x;
#endif
}
__host__ __device__ __forceinline__ double recip19(double x) { return 1.0 / x; }

// density deviation with one fixed summation order (for a node and for its neighbours)
template <typename R>
__host__ __device__ __forceinline__ R drho19(const R f[Q3]) {
    const R sf = ((f[1] + f[2]) + (f[3] + f[4])) + (f[5] + f[6]);
    const R se = (((f[7] + f[10]) + (f[8] + f[9])) + ((f[11] + f[14]) + (f[12] + f[13]))) +
                 ((f[15] + f[18]) + (f[16] + f[17]));
    return f[0] + (sf + se);
}

// Relaxation increments of the non-conserved modes for given noise xi[a] (a = 4..18), and
// the post-collision deviations o.  n[] holds xi (zero without noise).
template <typename R>
__host__ __device__ __forceinline__ void collide19(const Coef3<R>& a, const R f[Q3], const Rho3<R>& r,
                                                   const R xi[Q3], R o[Q3]) {
    const R c3 = R(1) / R(3), c6 = R(1) / R(6), c12 = R(1) / R(12);
    // Appendix B's stencils with the D3Q19 weights:
    // lap = sum_{i != 0} w_i [rho(r + c_i) + rho(r - c_i) - 2 rho(r)] / sigma_s^2
    //     = (1/3) sum_faces + (1/6) sum_edges - 4 rho(r);  d_a rho = 3 sum_i w_i c_ia rho(r + c_i)
    const R sfc = ((r.xp + r.xm) + (r.yp + r.ym)) + (r.zp + r.zm);
    const R sed = (((r.ap + r.am) + (r.bp + r.bm)) + ((r.cp + r.cm) + (r.dp + r.dm))) + ((r.ep + r.em) + (r.fp + r.fm));
    const R lap = sfc * c3 + sed * c6 - R(4) * r.c;
    const R ga = r.ap - r.am, gb = r.bp - r.bm, gc = r.cp - r.cm, gd = r.dp - r.dm, ge = r.ep - r.em,
            gf = r.fp - r.fm;
    const R gx = (r.xp - r.xm) * c6 + ((ga + gb) + (ge - gf)) * c12;
    const R gy = (r.yp - r.ym) * c6 + ((ga - gb) + (gc + gd)) * c12;
    const R gz = (r.zp - r.zm) * c6 + ((gc - gd) + (ge + gf)) * c12;

    // pair sums s and differences q of the opposite velocities
    const R sx = f[1] + f[2], qx = f[1] - f[2];
    const R sy = f[3] + f[4], qy = f[3] - f[4];
    const R sz = f[5] + f[6], qz = f[5] - f[6];
    const R sA = f[7] + f[10], qA = f[7] - f[10];
    const R sB = f[8] + f[9], qB = f[8] - f[9];
    const R sC = f[11] + f[14], qC = f[11] - f[14];
    const R sD = f[12] + f[13], qD = f[12] - f[13];
    const R sE = f[15] + f[18], qE = f[15] - f[18];
    const R sF = f[16] + f[17], qF = f[16] - f[17];
    const R sAB = sA + sB, sCD = sC + sD, sEF = sE + sF;
    const R sedge = (sAB + sCD) + sEF;
    const R sface = (sx + sy) + sz;

    // moments (rows of the basis): rho, j, bulk, shear, ghosts
    const R drho = f[0] + (sface + sedge);
    const R jx = qx + ((qA + qB) + (qE - qF));
    const R jy = qy + ((qA - qB) + (qC + qD));
    const R jz = qz + ((qC - qD) + (qE + qF));
    const R m4 = sedge - f[0];
    const R m5 = ((R(2) * sx - sy) - sz) + ((sAB + sEF) - R(2) * sCD);
    const R m6 = (sy - sz) + (sAB - sEF);
    const R m7 = sA - sB, m8 = sC - sD, m9 = sE - sF;
    const R m10 = ((qA + qB) + (qE - qF)) - R(2) * qx;
    const R m11 = ((qA - qB) + (qC + qD)) - R(2) * qy;
    const R m12 = ((qC - qD) + (qE + qF)) - R(2) * qz;
    const R m13 = (qA + qB) - (qE - qF);
    const R m14 = (qC + qD) - (qA - qB);
    const R m15 = (qE + qF) - (qC - qD);
    const R m16 = f[0] - R(2) * sface + sedge;
    const R m17 = ((sy + sz) - R(2) * sx) + ((sAB + sEF) - R(2) * sCD);
    const R m18 = (sz - sy) + (sAB - sEF);

    // equilibrium deviations
    const R rho = a.rho0 + drho;
    const R inv = recip19(rho);
    const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const R pxx = jx * ux + a.kappa * gx * gx;
    const R pyy = jy * uy + a.kappa * gy * gy;
    const R pzz = jz * uz + a.kappa * gz * gz;
    const R g2 = (gx * gx + gy * gy) + gz * gz;
    const R klap = a.kappa * rho * lap;
    const R dd = pressure_slope(a, drho);
    const R e4 = (dd * drho - R(3) * klap) + ((jx * ux + jy * uy) + jz * uz) - R(0.5) * a.kappa * g2;
    const R e5 = (R(2) * pxx - pyy) - pzz;
    const R e6 = pyy - pzz;
    const R e7 = jx * uy + a.kappa * gx * gy;
    const R e8 = jy * uz + a.kappa * gy * gz;
    const R e9 = jz * ux + a.kappa * gz * gx;
    const R e16 = (R(3) * klap - dd * drho) - R(4.5) * a.kappa * g2;

    // increments divided by N_a: D_a / N_a with D_a = lambda_a (m_a - m_a^eq) + xi_a
    const R h4 = R(1.5) * (a.lb * (m4 - e4) + xi[4]);
    const R h5 = R(0.75) * (a.ls * (m5 - e5) + xi[5]);
    const R h6 = R(2.25) * (a.ls * (m6 - e6) + xi[6]);
    const R h7 = R(9) * (a.ls * (m7 - e7) + xi[7]);
    const R h8 = R(9) * (a.ls * (m8 - e8) + xi[8]);
    const R h9 = R(9) * (a.ls * (m9 - e9) + xi[9]);
    const R h10 = R(1.5) * (a.lg * m10 + xi[10]);
    const R h11 = R(1.5) * (a.lg * m11 + xi[11]);
    const R h12 = R(1.5) * (a.lg * m12 + xi[12]);
    const R h13 = R(4.5) * (a.lg * m13 + xi[13]);
    const R h14 = R(4.5) * (a.lg * m14 + xi[14]);
    const R h15 = R(4.5) * (a.lg * m15 + xi[15]);
    const R h16 = R(0.5) * (a.lg * (m16 - e16) + xi[16]);
    const R h17 = R(0.75) * (a.lg * m17 + xi[17]);
    const R h18 = R(2.25) * (a.lg * m18 + xi[18]);

    // back to populations, w_i sum_a T_ai h_a: even part E (shared by a pair), odd part O
    const R wf = R(1) / R(18), we = R(1) / R(36);
    o[0] = f[0] + c3 * (h16 - h4);
    {
        const R E = wf * ((R(2) * h5 - R(2) * h16) - R(2) * h17), O = wf * (R(-2) * h10);
        o[1] = f[1] + (E + O);
        o[2] = f[2] + (E - O);
    }
    {
        const R E = wf * (((h6 - h5) - R(2) * h16) + (h17 - h18)), O = wf * (R(-2) * h11);
        o[3] = f[3] + (E + O);
        o[4] = f[4] + (E - O);
    }
    {
        const R E = wf * ((R(-1) * (h5 + h6) - R(2) * h16) + (h17 + h18)), O = wf * (R(-2) * h12);
        o[5] = f[5] + (E + O);
        o[6] = f[6] + (E - O);
    }
    // xy edges: common even part h4 + h5 + h6 + h16 + h17 + h18, +-h7
    const R exy = ((h4 + h16) + (h5 + h17)) + (h6 + h18);
    {
        const R E = we * (exy + h7), O = we * ((h10 + h11) + (h13 - h14));
        o[7] = f[7] + (E + O);
        o[10] = f[10] + (E - O);
    }
    {
        const R E = we * (exy - h7), O = we * ((h10 - h11) + (h13 + h14));
        o[8] = f[8] + (E + O);
        o[9] = f[9] + (E - O);
    }
    // yz edges: h4 - 2 h5 + h16 - 2 h17, +-h8
    const R eyz = (h4 + h16) - R(2) * (h5 + h17);
    {
        const R E = we * (eyz + h8), O = we * ((h11 + h12) + (h14 - h15));
        o[11] = f[11] + (E + O);
        o[14] = f[14] + (E - O);
    }
    {
        const R E = we * (eyz - h8), O = we * ((h11 - h12) + (h14 + h15));
        o[12] = f[12] + (E + O);
        o[13] = f[13] + (E - O);
    }
    // zx edges: h4 + h5 - h6 + h16 + h17 - h18, +-h9
    const R ezx = ((h4 + h16) + (h5 + h17)) - (h6 + h18);
    {
        const R E = we * (ezx + h9), O = we * ((h10 + h12) + (h15 - h13));
        o[15] = f[15] + (E + O);
        o[18] = f[18] + (E - O);
    }
    {
        const R E = we * (ezx - h9), O = we * ((h12 - h10) + (h13 + h15));
        o[16] = f[16] + (E + O);
        o[17] = f[17] + (E - O);
    }
}

}  // namespace lbf3
