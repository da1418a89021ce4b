/*
 * oracle/lbref.c -- plain FP64 CPU reference of the fluctuating D2Q9 step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header or table with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes follows Gross, Adhikari, Cates & Varnik, "Thermal
 * fluctuations in the lattice Boltzmann method for non-ideal fluids"
 * (arXiv:1009.0254):
 *   - the lattice Boltzmann equation in moment space, Eq. (gen-lbe-m), with the
 *     fluctuating collision of Eq. (fluct-lin-lbe): m*_a = m_a + lambda_a (m_a -
 *     m_a^eq) + xi_a, then f*_i = (T^-1 m*)_i and f_i(r + c_i, t+1) = f*_i(r, t);
 *   - the basis of Table I / Eq. (Tmat), built here from its polynomials;
 *   - the equilibrium moments of Table II with p0 = cs2 rho (linearised equation
 *     of state) or the bulk pressure of the Landau double well of Sec. II A, no
 *     Galilean corrections (C_n = 0) and no forcing (m^F = 0);
 *   - the Laplacian of Appendix B and the isotropic gradient
 *     d_alpha rho = 3 sum_i w_i c_i,alpha rho(r + c_i) for the (grad rho)^2 terms.
 * The noise xi_a(r) is an input (the Python side builds it per Sec. IV).
 *
 * Random numbers: Philox4x32-10 of Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11), and the Box-Muller transform; the
 * counter layout is documented at oracle_normals().
 *
 * Layout of every population array: f[i][y][x] -> f[i*nx*ny + y*nx + x], FP64,
 * pre-collision populations (the state right after streaming).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

static int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};   /* c_OPP[i] = -c_i */
static double WT[Q];
static double TM[Q][Q];    /* T[a][i] */
static double NA[Q];       /* N_a */
static double TI[Q][Q];    /* (T^-1)[i][a] */
static int ready = 0;

static void init_tables(void) {
    if (ready) return;
    for (int i = 0; i < Q; ++i) {
        WT[i] = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        double cx = CX[i], cy = CY[i], c2 = cx * cx + cy * cy;
        TM[0][i] = 1.0;
        TM[1][i] = cx;
        TM[2][i] = cy;
        TM[3][i] = 3.0 * c2 - 2.0;
        TM[4][i] = 2.0 * cx * cx - c2;
        TM[5][i] = cx * cy;
        TM[6][i] = (3.0 * c2 - 4.0) * cx;
        TM[7][i] = (3.0 * c2 - 4.0) * cy;
        TM[8][i] = 9.0 * c2 * c2 - 15.0 * c2 + 2.0;
    }
    for (int a = 0; a < Q; ++a) {
        NA[a] = 0.0;
        for (int i = 0; i < Q; ++i) NA[a] += WT[i] * TM[a][i] * TM[a][i];
    }
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < Q; ++a) TI[i][a] = WT[i] * TM[a][i] / NA[a];
    ready = 1;
}

/* Exposes the tables for the tests (T[a][i] row-major, N[a], w[i], c[i][2]). */
void oracle_tables(double* T_out, double* N_out, double* w_out, int* c_out) {
    init_tables();
    for (int a = 0; a < Q; ++a)
        for (int i = 0; i < Q; ++i) T_out[a * Q + i] = TM[a][i];
    for (int a = 0; a < Q; ++a) N_out[a] = NA[a];
    for (int i = 0; i < Q; ++i) {
        w_out[i] = WT[i];
        c_out[2 * i] = CX[i];
        c_out[2 * i + 1] = CY[i];
    }
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 Philox S-box,  */
/* round multipliers 0xD2511F53 and 0xCD9E8D57, key schedule Weyl increments   */
/* 0x9E3779B9 and 0xBB67AE85 added between rounds.                             */
/* ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One output word -> one Box-Muller pair.  The top 20 bits give the radius uniform
 * u1 = (k + 1/2) 2^-20, the low 12 bits the angle uniform u2 = (j + 1/2) 2^-12; both are
 * exact in FP32 as well as FP64.  Then (u1, u2) -> sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2):
 * |n| <= sqrt(-2 ln 2^-21) = 5.39, and the 4096 equally spaced angles keep every moment of
 * the pair below order 4096 exact. */
static void box_muller_word(uint32_t w, double* n0, double* n1) {
    const double two_pi = 6.283185307179586476925286766559;
    const double u1 = ((double)(w >> 12) + 0.5) * (1.0 / 1048576.0);
    const double u2 = ((double)(w & 0xfffu) + 0.5) * (1.0 / 4096.0);
    const double r = sqrt(-2.0 * log(u1));
    *n0 = r * cos(two_pi * u2);
    *n1 = r * sin(two_pi * u2);
}

/*
 * Eight unit normals per entry of `index[]` for one (seed, step, tag):
 *   key     = (seed & 0xffffffff, seed >> 32)
 *   counter = (index, step & 0xffffffff, step >> 32, tag)
 *   normals = the Box-Muller pairs of output words 0, 1, 2, 3 in that order.
 * index is the node number y*nx + x (or a wavevector number), tag selects the draw:
 * 0 -> per node: words 0, 1 -> nu_5..nu_8, word 2 -> (nu_4, nu_9);
 * 2 -> k-space eta from words 0, 1.
 * out[8*j + q] receives normal q of entry j.
 */
void oracle_normals(int64_t count, const uint32_t* index, uint64_t seed, uint64_t step,
                    uint32_t tag, double* out) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int64_t j = 0; j < count; ++j) {
        uint32_t ctr[4] = {index[j], (uint32_t)(step & 0xffffffffu), (uint32_t)(step >> 32), tag};
        uint32_t r[4];
        oracle_philox4x32_10(ctr, key, r);
        for (int q = 0; q < 4; ++q) box_muller_word(r[q], &out[8 * j + 2 * q], &out[8 * j + 2 * q + 1]);
    }
}

/* ------------------------------------------------------------------------- */
/* Collision at one site (Eq. fluct-lin-lbe, Table II, Appendix B).           */
/* ------------------------------------------------------------------------- */
typedef struct {
    double rho0, cs2, kappa;
    double lam[Q];
    int eos;                       /* 0: p0 = cs2 rho;  1: Landau double well (Sec. II A) */
    double beta, rhoV, rhoL;       /* f0 = beta (rho - rhoV)^2 (rho - rhoL)^2 */
} params_t;

/* Bulk pressure of the equation of state (Sec. II A): p0 = rho d(f0)/d(rho) - f0 for the
 * double well f0 = beta (rho - rhoV)^2 (rho - rhoL)^2, else the linearised p0 = cs2 rho. */
static double bulk_pressure(const params_t* p, double rho) {
    if (p->eos == 1) {
        const double a = rho - p->rhoV, b = rho - p->rhoL;
        const double f0 = p->beta * a * a * b * b;
        const double df0 = 2.0 * p->beta * a * b * (a + b);          /* d f0 / d rho */
        return rho * df0 - f0;
    }
    return p->cs2 * rho;
}

static int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

/* rho_nb[j] = rho(r + c_j), j = 0..8 (j = 0 is the site itself); f[i] = f_i(r);
 * xi[a] = noise of mode a; fstar[i] receives the post-collision populations. */
static void collide_site(const params_t* p, const double rho_nb[Q], const double f[Q],
                         const double xi[Q], double fstar[Q]) {
    const double s2 = 1.0 / 3.0;
    double m[Q], meq[Q], ms[Q];
    for (int a = 0; a < Q; ++a) {
        m[a] = 0.0;
        for (int i = 0; i < Q; ++i) m[a] += TM[a][i] * f[i];
    }
    double rho = m[0], jx = m[1], jy = m[2];
    double ux = jx / rho, uy = jy / rho;

    /* Appendix B Laplacian and the isotropic gradient, on rho at r + c_j */
    double lap = 0.0, gx = 0.0, gy = 0.0;
    for (int j = 1; j < Q; ++j) {
        /* sum over i != 1 of w_i [rho(r+c_i) + rho(r-c_i) - 2 rho(r)] / sigma_s^2 */
        lap += WT[j] * (rho_nb[j] + rho_nb[OPP[j]] - 2.0 * rho_nb[0]) / s2;
        gx += 3.0 * WT[j] * CX[j] * rho_nb[j];
        gy += 3.0 * WT[j] * CY[j] * rho_nb[j];
    }
    double p0 = bulk_pressure(p, rho);                          /* equation of state */
    double iso = p0 - rho * s2 - p->kappa * rho * lap;
    meq[0] = rho;
    meq[1] = rho * ux;
    meq[2] = rho * uy;
    meq[3] = 3.0 * rho * (ux * ux + uy * uy) + 6.0 * iso;
    meq[4] = rho * (ux * ux - uy * uy) + p->kappa * (gx * gx - gy * gy);
    meq[5] = rho * ux * uy + p->kappa * gx * gy;
    meq[6] = 0.0;
    meq[7] = 0.0;
    meq[8] = -6.0 * iso - 3.0 * p->kappa * (gx * gx + gy * gy);

    for (int a = 0; a < Q; ++a) ms[a] = m[a] + p->lam[a] * (m[a] - meq[a]) + xi[a];
    for (int i = 0; i < Q; ++i) {
        fstar[i] = 0.0;
        for (int a = 0; a < Q; ++a) fstar[i] += TI[i][a] * ms[a];
    }
}

static void load_params(params_t* p, const double* par) {
    /* par = {rho0, cs2, kappa, lambda_1 .. lambda_9, eos, beta, rhoV, rhoL} */
    p->rho0 = par[0];
    p->cs2 = par[1];
    p->kappa = par[2];
    for (int a = 0; a < Q; ++a) p->lam[a] = par[3 + a];
    p->eos = (int)par[12];
    p->beta = par[13];
    p->rhoV = par[14];
    p->rhoL = par[15];
}

/*
 * One full step: collide at every site with noise xi[a][y][x] (NULL = no noise),
 * then stream f_i(r + c_i) = f*_i(r) with periodic wrap.  fin and fout must not
 * alias.
 */
void oracle_step(int nx, int ny, const double* fin, double* fout, const double* par,
                 const double* xi) {
    init_tables();
    params_t p;
    load_params(&p, par);
    const int64_t n = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t s = 0; s < n; ++s) {
        double r = 0.0;
        for (int i = 0; i < Q; ++i) r += fin[i * n + s];
        rho[s] = r;
    }
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            double rho_nb[Q], f[Q], xs[Q], fs[Q];
            for (int j = 0; j < Q; ++j)
                rho_nb[j] = rho[(int64_t)wrap(y + CY[j], ny) * nx + wrap(x + CX[j], nx)];
            for (int i = 0; i < Q; ++i) f[i] = fin[i * n + s];
            for (int a = 0; a < Q; ++a) xs[a] = xi ? xi[a * n + s] : 0.0;
            collide_site(&p, rho_nb, f, xs, fs);
            for (int i = 0; i < Q; ++i) {
                int64_t d = (int64_t)wrap(y + CY[i], ny) * nx + wrap(x + CX[i], nx);
                fout[i * n + d] = fs[i];
            }
        }
    }
    free(rho);
}

/*
 * Post-collision populations at selected sites only (for sampled comparisons on
 * lattices too large to step on the CPU): site k is sites[k] = y*nx + x, its noise
 * is xi_sites[9*k + a], and fstar[9*k + i] receives f*_i at that site.
 */
void oracle_collide_sites(int nx, int ny, const double* fin, int64_t nsites,
                          const int64_t* sites, const double* par, const double* xi_sites,
                          double* fstar) {
    init_tables();
    params_t p;
    load_params(&p, par);
    const int64_t n = (int64_t)nx * ny;
    for (int64_t k = 0; k < nsites; ++k) {
        int64_t s = sites[k];
        int x = (int)(s % nx), y = (int)(s / nx);
        double rho_nb[Q], f[Q], xs[Q];
        for (int j = 0; j < Q; ++j) {
            int64_t t = (int64_t)wrap(y + CY[j], ny) * nx + wrap(x + CX[j], nx);
            double r = 0.0;
            for (int i = 0; i < Q; ++i) r += fin[i * n + t];
            rho_nb[j] = r;
        }
        for (int i = 0; i < Q; ++i) f[i] = fin[i * n + s];
        for (int a = 0; a < Q; ++a) xs[a] = xi_sites ? xi_sites[Q * k + a] : 0.0;
        collide_site(&p, rho_nb, f, xs, &fstar[Q * k]);
    }
}
