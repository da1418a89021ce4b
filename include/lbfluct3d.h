/*
 * lbfluct3d.h -- C ABI of the three-dimensional members (D3Q19, D3Q27) of the GB300 (sm_103a)
 * fluctuating lattice Boltzmann library.
 *
 * [GACV] = Gross, Adhikari, Cates & Varnik, "Thermal fluctuations in the lattice Boltzmann
 * method for non-ideal fluids", arXiv:1009.0254.  Sec. IV states that its construction of
 * the noise from the lattice fluctuation-dissipation theorem holds on any DdQn lattice;
 * these entry points step the same non-ideal model on a periodic nx x ny x nz lattice:
 *   - collision: [GACV] Eq. (fluct-lin-lbe), m*_a = m_a + lambda_a (m_a - m_a^eq) + xi_a, with
 *     lambda_b = -1/tau_b on the bulk mode, lambda_s = -1/tau_s on the traceless second-order
 *     modes and -1/tau_ghost on every higher mode;
 *   - equilibrium: rho, j and the second moments of P^th + rho u u, with P^th the pressure
 *     tensor of [GACV] Eq. (press-ten) for p0 = cs2 rho, i.e.
 *     sum_i f^eq_i c_ia c_ib = (p0 - kappa rho lap rho - kappa |grad rho|^2 / 2) delta_ab
 *     + kappa d_a rho d_b rho + rho u_a u_b; lap and grad are the isotropic stencils of
 *     [GACV] Appendix B with the lattice's weights; the ghost equilibria below make a field
 *     that is uniform along one axis evolve, at equal relaxation times, as the D2Q9 model of
 *     [GACV] Table II;
 *   - noise: spatially uncorrelated with covariance Xi(0) of [GACV] Eq. (noise-matrix-k0),
 *     xi = L nu, L the Cholesky factor of the block of the non-conserved modes (LB_NOISE_LW);
 *     or spatially correlated with covariance Xi(k) of [GACV] Eq. (noise-matrix) at every k
 *     (LB_NOISE_FULL_RS): with the ansatz of Eq. (f-correl-yeo) the advection drops out of the
 *     fluctuation-dissipation relation, so Xi(k) is Xi(0) at c_s^2(k) = cs2 + rho0 kappa s(k)
 *     (Eq. sound-speed-k, s the Laplacian symbol); only the coupled block (D3Q19 the modes 4
 *     and 16, D3Q27 the seven listed below) depends on k, affinely in s, and s is multilinear
 *     in (cos kx, cos ky, cos kz), so Xi(k) is the multilinear interpolation of its values at
 *     the corners k in {0, pi}^3 (s = 0, 4, 16/3, 4 on D3Q19 and 0, 4, 16/3, 52/9 on D3Q27 for
 *     0..3 components at pi).  Eight white vector fields nu_abc per node (a, b, c = +-1; +1
 *     for k = 0), each times a factor L_abc with L_abc L_abc^T the value at its corner of the
 *     part built in real space, combined as h_d(r) = (1/8) sum_abc a^dx b^dy c^dz L_abc
 *     nu_abc(r), give the noise sum over d in {0,1}^3 of h_d(r - d), whose covariance is the
 *     multilinear interpolation of the corner values.  D3Q19: the whole (4,16) block, L_abc its
 *     Cholesky factor at the corner.  D3Q27: the block is X0 + s(k) D with D = p p^T - q q^T
 *     of rank two (the slope of Xi(0) in c_s^2), so it is C + s(k) p p^T + (S - s(k)) q q^T,
 *     S = 52/9 and C = X0 - S q q^T: a white part with factor chol(C) (on the long-wavelength
 *     normals of the coupled modes) plus p phi_p + q phi_q, the scalar fields phi_p, phi_q
 *     built as above with the corner amplitudes sqrt(s) and sqrt(S - s); p and q come from the
 *     eigenvectors of L0^-1 D L0^-T (X0 = L0 L0^T), the split for which C is positive
 *     semidefinite exactly when the block at s = S is, and the first component of p (of q) of
 *     magnitude at least half its largest is positive.  The covariance is exactly Xi(k); Xi
 *     must be positive semidefinite at the corner values (D3Q27: at s = 0 and s = S, with the
 *     block at s = 0 positive definite).  The other modes as LB_NOISE_LW;
 *     or spatially uncorrelated with Xi(0) of a homogeneous system at each node's own density
 *     rho(r) and sound speed c_s^2(rho(r)) (LB_NOISE_LW_LOCAL, Sec. IV and Sec. V B for
 *     inhomogeneous systems): Xi(0) is rho (A + B c_s^2) entrywise, the coupled block is
 *     factored at every node by Cholesky with a negative pivot clamped to zero (where the local
 *     block is not positive semidefinite), the other modes scale with sqrt(rho); the draws are
 *     those of LB_NOISE_LW, and at uniform density the two modes give the same noise;
 *   - equation of state: p0 = cs2 rho, or the Landau double well of [GACV] Sec. II A
 *     (lb3_set_eos), whose bulk pressure enters the second moments and the ghost equilibria.
 *
 * LB_D3Q19 (19 velocities, weights 1/3, 1/18, 1/36)
 *   - modes: the weighted-orthogonal basis of Duenweg, Schiller & Ladd, Phys. Rev. E 76,
 *     036704 (2007), Table I (m_0 = rho, m_1..3 = j, m_4 = bulk c^2 - 1, m_5..9 shear,
 *     m_10..18 ghosts); only m_16 = 3c^4 - 6c^2 + 1 among the ghosts has an equilibrium,
 *     m_16^eq = -3 (p0 - rho/3 - kappa rho lap rho) - (9/2) kappa |grad rho|^2;
 *   - velocity order: 0 rest; 1 (1,0,0), 2 (-1,0,0), 3 (0,1,0), 4 (0,-1,0), 5 (0,0,1),
 *     6 (0,0,-1); 7 (1,1,0), 8 (1,-1,0), 9 (-1,1,0), 10 (-1,-1,0); 11 (0,1,1), 12 (0,1,-1),
 *     13 (0,-1,1), 14 (0,-1,-1); 15 (1,0,1), 16 (-1,0,1), 17 (1,0,-1), 18 (-1,0,-1);
 *   - random numbers: tag 4 gives nu_4..nu_11, tag 5 gives nu_12..nu_18; xi_a = sqrt(Xi_aa) nu_a
 *     except xi_4 = L_44 nu_4, xi_16 = L_16,4 nu_4 + L_16,16 nu_16 (LB_NOISE_LW); the corner
 *     fields of LB_NOISE_FULL_RS from tags 10 and 11, word w of the pair giving nu of corner
 *     w = 4 ia + 2 ib + ic (index 0: sign +1).
 * LB_D3Q27 (27 velocities, weights the products of the D1Q3 weights 2/3, 1/6, 1/6)
 *   - velocity i = 9 ix + 3 iy + iz with c = (v[ix], v[iy], v[iz]), v = (0, 1, -1);
 *   - modes: the products m_(a,b,c) = sum_i p_a(c_ix) p_b(c_iy) p_c(c_iz) f_i of p_0 = 1,
 *     p_1 = c, p_2 = 3c^2 - 1 (mode index 9a + 3b + c; the c_z-independent modes are the D2Q9
 *     basis of [GACV] Table I); ghost equilibria p_2a p_2b = -3 (p0 - rho/3 - kappa rho lap rho)
 *     - (3/2) kappa |grad rho|^2, p_2x p_2y p_2z = 3 (p0 - rho/3 - kappa rho lap rho)
 *     - (3/2) kappa |grad rho|^2, all others zero;
 *   - random numbers: tags 6, 7, 8 give 24 normals, the n-th going to the n-th non-conserved
 *     mode in mode order; the factor is diagonal except on the modes p_2z, p_2y, p_2y p_2z,
 *     p_2x, p_2x p_2z, p_2x p_2y, p_2x p_2y p_2z, which share a dense Cholesky block (the
 *     coupled block); the corner fields of LB_NOISE_FULL_RS from tags 12 and 13, word w of the
 *     pair giving (nu of phi_p, nu of phi_q) of corner w = 4 ia + 2 ib + ic.
 *
 * Conventions
 *   - Return codes and buffer locations are those of lbfluct.h (LB_OK, LB_E*, LB_HOST,
 *     LB_DEVICE, LB_FP32, LB_FP64, LB_NOISE_OFF, LB_NOISE_LW).
 *   - Populations cross the ABI as FP64 arrays f[i][z][y][x] (index
 *     ((i*nz + z)*ny + y)*nx + x), pre-collision (right after streaming), in the lattice's
 *     velocity order above.
 *   - The device holds the deviations f_i - fbar_i from the rest state in the storage
 *     precision (LB_FP32: 2 Q 4 bytes moved per node update; LB_FP64: 2 Q 8), two copies,
 *     each plane with periodic ghost copies of 32 bytes of elements on either side of a row
 *     and two rows below and above every z plane.
 *   - Philox4x32-10 keyed (seed mod 2^32, seed div 2^32), counter (node, t mod 2^32,
 *     t div 2^32, tag) with node = (z*ny + y)*nx + x; one Box-Muller pair per output word
 *     (20-bit radius, 12-bit angle, as for D2Q9).
 *   - All GPU work runs on the context's stream; calls that return data synchronise it.
 *     A step kernel whose bounded wait for its staged loads gave up is reported as LB_ETIMEOUT
 *     by the next lb3_synchronize, lb3_get_populations or lb3_sums (the word is then cleared).
 *     The caller owns every buffer it passes.  One host thread per context at a time.
 */
#ifndef LBFLUCT3D_H
#define LBFLUCT3D_H

#include <stddef.h>
#include <stdint.h>

#include "lbfluct.h"

#ifdef __cplusplus
extern "C" {
#endif

/* lattices */
#define LB_D3Q19 19
#define LB_D3Q27 27

typedef struct lb3_ctx lb3_ctx;

/* Device bytes of a context (two population copies with their ghost copies, FP64 staging
 * plane, reduction scratch, error word); 0 for invalid sizes, lattice or precision. */
size_t lb3_workspace_bytes(int nx, int ny, int nz, int lattice, int precision);

/*
 * Creates a context for a periodic nx x ny x nz lattice (each >= 1, nx*ny*nz < 2^32) of the
 * given kind (LB_D3Q19 or LB_D3Q27) at rest with density rho0: fbar_i = w_i 3 cs2 rho0 for
 * the moving velocities and the remainder rho0 - sum on the rest velocity (the equilibrium
 * at u = 0 for p0 = cs2 rho).  precision: LB_FP32 or LB_FP64 (LB_EINVAL otherwise).  The
 * library allocates its device memory (LB_ENOMEM if that fails).  *out receives the context.
 */
int lb3_create(int nx, int ny, int nz, int lattice, int precision, uint64_t seed, double rho0, double cs2,
               lb3_ctx** out);
int lb3_destroy(lb3_ctx* ctx);
int lb3_set_stream(lb3_ctx* ctx, void* stream);

/*
 * Sets kT, kappa, the relaxation times (each > 1/2) and the noise mode (LB_NOISE_OFF,
 * LB_NOISE_LW, LB_NOISE_FULL_RS or LB_NOISE_LW_LOCAL; others LB_EINVAL).  With LB_NOISE_LW or
 * LB_NOISE_FULL_RS and kT > 0, the c_s^2 of the linear theory about rho0 must be positive and
 * Xi(0) (with LB_NOISE_FULL_RS also Xi at the other corner values of s) positive semidefinite
 * (D3Q19 at equal relaxation times: c_s^2 <= 5/9; D3Q27 with LB_NOISE_FULL_RS: the coupled
 * block positive definite at s = 0 and positive semidefinite at s = 52/9), else LB_ENOTPSD.  May be called again between
 * steps; the lattice state is kept.
 */
int lb3_set_params(lb3_ctx* ctx, double kT, double kappa, double tau_s, double tau_b, double tau_ghost,
                   int noise_mode);

/*
 * Equation of state, [GACV] Sec. II A, as lb_set_eos of lbfluct.h: LB_EOS_LINEAR restores
 * p0 = cs2 rho with the cs2 of lb3_create; LB_EOS_DOUBLE_WELL takes p0 = rho df0/drho - f0 of
 * f0 = beta (rho - rhoV)^2 (rho - rhoL)^2 (beta > 0, 0 <= rhoV < rhoL) at every node, as the
 * exact quartic in rho - rho0.  The uniform rest state becomes the equilibrium at rho0 with
 * p0(rho0); the linear theory about rho0 that sets LB_NOISE_LW and LB_NOISE_FULL_RS takes
 * c_s^2 = rho0 d2f0/drho2 (rho0), and LB_NOISE_LW_LOCAL takes c_s^2(rho(r)) at every node.  The
 * populations are kept (their stored deviations are re-based on the new rest state) and the
 * parameters of the last lb3_set_params re-applied (its error, if the new linear theory
 * refuses them).  LB_EINVAL for bad arguments.
 */
int lb3_set_eos(lb3_ctx* ctx, int eos, double beta, double rhoV, double rhoL);

/* Advances nsteps time steps (one kernel launch each); asynchronous. */
int lb3_step(lb3_ctx* ctx, int64_t nsteps);
int lb3_get_time(lb3_ctx* ctx, int64_t* t);

/* Writes / reads all Q populations (FP64, layout above) at `loc`; set also sets the time t
 * (the index of the next collision, which keys its random numbers). */
int lb3_set_populations(lb3_ctx* ctx, const double* f, int loc, int64_t t);
int lb3_get_populations(lb3_ctx* ctx, double* f, int loc);

/* sums[0] = total mass, sums[1..3] = total momentum (FP64 accumulation of the deviations
 * plus the rest state's share). */
int lb3_sums(lb3_ctx* ctx, double sums[4]);

/* CUDA-event timing of every `every`-th step-kernel launch on the context's stream (0 off;
 * setting resets the totals); lb3_kernel_time returns the summed milliseconds and the
 * number of timed launches. */
int lb3_set_kernel_timing(lb3_ctx* ctx, int every);
int lb3_kernel_time(lb3_ctx* ctx, double* ms, int64_t* launches);
/* Kernels launched on behalf of the context so far. */
int lb3_launch_count(lb3_ctx* ctx, int64_t* launches);
int lb3_synchronize(lb3_ctx* ctx);
const char* lb3_last_error(lb3_ctx* ctx);

/* Host-side FP64 Xi(0) of the lattice's model (Q x Q, row-major, in its mode order) for these
 * parameters; LB_EINVAL for an unknown lattice or parameters out of range. */
int lb3_noise_matrix(int lattice, double rho0, double cs2, double kT, double tau_s, double tau_b,
                     double tau_ghost, double* xi);

#ifdef __cplusplus
}
#endif

#endif /* LBFLUCT3D_H */
