// lb3d.cu -- host side of the D3Q19 and D3Q27 lattices and the C ABI of lbfluct3d.h: the
// lattices' Xi(0) and its factors, the padded population storage (lb3d_kernel.cuh) and its
// transfers, the choice of the step kernel, and the tensor maps of its TMA staging.  The
// step kernels are compiled in lb3d_q19.cu and lb3d_q27.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "lb3d_kernel.cuh"
#include "lbfluct3d.h"

namespace lbf3 {

constexpr double SIGMA_S2 = 1.0 / 3.0;

// ---- host-side theory --------------------------------------------------------------------

static double w_of(int lattice, int i) { return lattice == 19 ? Lat19::w(i) : Lat27::w(i); }
static int c_of(int lattice, int i, int k) { return lattice == 19 ? Lat19::c(i, k) : Lat27::c(i, k); }
// the stored plane of population i
static int sigma_of(int lattice, int i) { return lattice == 19 ? Lat19::sigma(i) : Lat27::sigma(i); }

// rest populations of bulk pressure p0: w_i 3 p0 on the moving velocities, the remainder at
// rest (p0 = cs2 rho0 for the linearised equation of state)
static void rest_pops(int lattice, double rho0, double p0, double* fbar) {
    double moving = 0.0;
    for (int i = 1; i < lattice; ++i) {
        fbar[i] = w_of(lattice, i) * 3.0 * p0;
        moving += fbar[i];
    }
    fbar[0] = rho0 - moving;
}

static double norm19(int a) {
    static const double N[Q3] = {1, 1.0 / 3, 1.0 / 3, 1.0 / 3, 2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                 2.0 / 3, 2.0 / 3, 2.0 / 3, 2.0 / 9, 2.0 / 9, 2.0 / 9, 2.0, 4.0 / 3, 4.0 / 9};
    return N[a];
}

// D3Q19 Xi(0) in closed form: in the variables y4 = m4 - d rho, y16 = m16 + d rho
// (d = 3 cs2 - 1) the linearised collision is diagonal and the equal-time covariances of the
// ansatz <df_i df_j> = (S/rho0) fbar_i delta_ij (S = rho0 kT / cs2) are rho0 kT (5 - 9 cs2),
// 9 rho0 kT (1 - cs2), 3 rho0 kT (3 cs2 - 1) for (y4, y4), (y16, y16), (y4, y16) and
// N_a rho0 kT / sigma_s^2 for the other non-conserved modes; stationarity under
// m -> (1 + lambda) m + xi gives the entries below.
static void xi_zero19(double rho0, double cs2, double kT, double lb, double ls, double lg, double* X) {
    for (int k = 0; k < Q3 * Q3; ++k) X[k] = 0.0;
    auto til = [](double l) { return l * (2.0 + l); };
    for (int a = 5; a < Q3; ++a) {
        const double l = a <= 9 ? ls : lg;
        X[a * Q3 + a] = -(rho0 * kT / SIGMA_S2) * norm19(a) * til(l);
    }
    X[4 * Q3 + 4] = -rho0 * kT * (5.0 - 9.0 * cs2) * til(lb);
    X[16 * Q3 + 16] = -9.0 * rho0 * kT * (1.0 - cs2) * til(lg);
    X[4 * Q3 + 16] = X[16 * Q3 + 4] = -3.0 * rho0 * kT * (3.0 * cs2 - 1.0) * (lb + lg + lb * lg);
}

// D3Q27 Xi(0).  The rest populations are fbar_i = 3 cs2 rho0 w_i + rho0 (1 - 3 cs2) delta_i0,
// so the ansatz covariance is the rank-one update G = S [3 cs2 diag(N) + (1 - 3 cs2) t0 t0^T]
// (t0: the modes at c = 0, S = rho0 kT / cs2).  With y = (I - J) m (J the density
// dependence of the equilibrium at rest) the ansatz makes y uncorrelated with rho, so the
// fluctuation-dissipation relation of Eq. (noise-matrix-k0) becomes
// Xi = -(Y Lambda^T + Lambda Y + Lambda Y Lambda^T) with Y = (I - J) G (I - J)^T.
static void xi_zero27(double rho0, double cs2, double kT, double lb, double ls, double lg, double* X) {
    constexpr int Q = Q27;
    const double n1[3] = {1.0, 1.0 / 3.0, 2.0};
    auto p0 = [](int a) { return a == 0 ? 1.0 : (a == 1 ? 0.0 : -1.0); };   // p_a at c = 0
    std::vector<double> N(Q), t0(Q), G(Q * Q), A(Q * Q, 0.0), Lm(Q * Q, 0.0), Y(Q * Q, 0.0), tmp(Q * Q, 0.0);
    for (int k = 0; k < Q; ++k) {
        N[k] = n1[k / 9] * n1[(k / 3) % 3] * n1[k % 3];
        t0[k] = p0(k / 9) * p0((k / 3) % 3) * p0(k % 3);
    }
    const double S = rho0 * kT / cs2, d = 3.0 * cs2 - 1.0;
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b)
            G[a * Q + b] = S * ((a == b ? 3.0 * cs2 * N[a] : 0.0) + (1.0 - 3.0 * cs2) * t0[a] * t0[b]);
    auto conserved = [](int k) { return k == 0 || k == 1 || k == 3 || k == 9; };
    for (int k = 0; k < Q; ++k) A[k * Q + k] = conserved(k) ? 0.0 : 1.0;
    for (int k : {2, 6, 18, 26}) A[k * Q + 0] = -d;          // p_2a and the sixth order follow +d rho
    for (int k : {8, 20, 24}) A[k * Q + 0] = d;              // p_2a p_2b follow -d rho
    for (int k = 0; k < Q; ++k)
        if (!conserved(k)) Lm[k * Q + k] = lg;
    for (int k : {4, 10, 12}) Lm[k * Q + k] = ls;
    for (int a : {2, 6, 18})
        for (int b : {2, 6, 18}) Lm[a * Q + b] = (lb - ls) / 3.0 + (a == b ? ls : 0.0);
    for (int a = 0; a < Q; ++a)           // tmp = A G
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;
            for (int c = 0; c < Q; ++c) s += A[a * Q + c] * G[c * Q + b];
            tmp[a * Q + b] = s;
        }
    for (int a = 0; a < Q; ++a)           // Y = A G A^T
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;
            for (int c = 0; c < Q; ++c) s += tmp[a * Q + c] * A[b * Q + c];
            Y[a * Q + b] = s;
        }
    std::vector<double> LY(Q * Q, 0.0);   // Lambda Y
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;
            for (int c = 0; c < Q; ++c) s += Lm[a * Q + c] * Y[c * Q + b];
            LY[a * Q + b] = s;
        }
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;               // (Lambda Y Lambda^T)_ab
            for (int c = 0; c < Q; ++c) s += LY[a * Q + c] * Lm[b * Q + c];
            X[a * Q + b] = -(LY[b * Q + a] + LY[a * Q + b] + s);
        }
}

// lower-triangular Cholesky of the block idx[] of X (row-major, leading dimension Q); pivots
// that are zero up to 1e-12 of the block's scale are clamped; false for a negative pivot
static bool cholesky_block(const double* X, int Q, const std::vector<int>& idx, std::vector<double>& L) {
    const int n = (int)idx.size();
    L.assign((size_t)n * n, 0.0);
    double scale = 1e-300;
    for (int k : idx) scale = std::max(scale, std::fabs(X[k * Q + k]));
    for (int j = 0; j < n; ++j) {
        double s = X[idx[j] * Q + idx[j]];
        for (int q = 0; q < j; ++q) s -= L[j * n + q] * L[j * n + q];
        if (s <= 1e-12 * scale) {
            if (s < -1e-9 * scale) return false;
            continue;
        }
        L[j * n + j] = std::sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = X[idx[i] * Q + idx[j]];
            for (int q = 0; q < j; ++q) t -= L[i * n + q] * L[j * n + q];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    return true;
}

// Eigenvalues (ascending, w) and orthonormal eigenvectors (the columns of V, row-major) of a
// symmetric n x n matrix A by cyclic Jacobi rotations (each zeroes one off-diagonal pair; the
// sweeps repeat until the off-diagonal part vanishes to rounding).
static void sym_eigen(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    double scale = 0.0;
    for (double v : A) scale = std::max(scale, std::fabs(v));
    for (int sweep = 0; sweep < 100 && scale > 0.0; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off = std::max(off, std::fabs(A[i * n + j]));
        if (off <= 1e-17 * scale) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (std::fabs(apq) <= 1e-300) continue;
                const double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {        // A <- A J (columns p, q)
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {        // A <- J^T A (rows p, q)
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {        // V <- V J
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return A[x * n + x] < A[y * n + y]; });
    std::vector<double> W((size_t)n * n);
    w.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        w[j] = A[ord[j] * n + ord[j]];
        for (int i = 0; i < n; ++i) W[i * n + j] = V[i * n + ord[j]];
    }
    V = W;
}

// D3Q27 correlated noise: the coupled block of Xi(k) is X0 + s(k) D with D of rank two (the
// slope of Xi(0) in c_s^2 times rho0 kappa), so with S = 52/9 (the largest s) and
// D = p p^T - q q^T it is C + s p p^T + (S - s) q q^T, C = X0 - S q q^T.  The split that
// whitens X0 (X0 = L0 L0^T, L0^-1 D L0^-T = mu+ y+ y+^T + mu- y- y-^T, p = sqrt(mu+) L0 y+,
// q = sqrt(-mu-) L0 y-) makes C = L0 (I - S |mu-| y- y-^T) L0^T positive semidefinite exactly
// when X at k = (pi, pi, pi) is.  Signs: the first component of p (of q) of magnitude at least
// half its largest is positive.  Out: Lw the Cholesky factor of C (row-major 7 x 7), p, q;
// false where X0 is singular, D is not of that form or C is indefinite.
static bool rs_split27(double rho0, double cs2, double kappa, double kT, double lb, double ls, double lg,
                       std::vector<double>& Lw, double p[7], double q[7]) {
    constexpr int n = 7;
    const double S = 52.0 / 9.0;
    const std::vector<int> coupled(COUPLED27, COUPLED27 + 7);
    std::vector<double> X((size_t)27 * 27), XS((size_t)27 * 27);
    xi_zero27(rho0, cs2, kT, lb, ls, lg, X.data());
    xi_zero27(rho0, cs2 + rho0 * kappa * S, kT, lb, ls, lg, XS.data());
    std::vector<double> X0((size_t)n * n), D((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            X0[i * n + j] = X[coupled[i] * 27 + coupled[j]];
            D[i * n + j] = (XS[coupled[i] * 27 + coupled[j]] - X0[i * n + j]) / S;
        }
    std::vector<double> L0;
    const std::vector<int> all = {0, 1, 2, 3, 4, 5, 6};
    if (!cholesky_block(X0.data(), n, all, L0)) return false;
    for (int i = 0; i < n; ++i)
        if (!(L0[i * n + i] > 0.0)) return false;
    // Y = L0^-1 D L0^-T: forward substitution on the columns of D, then on the rows
    std::vector<double> Z((size_t)n * n), Y((size_t)n * n);
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double t = D[i * n + c];
            for (int k = 0; k < i; ++k) t -= L0[i * n + k] * Z[k * n + c];
            Z[i * n + c] = t / L0[i * n + i];
        }
    for (int r = 0; r < n; ++r)
        for (int i = 0; i < n; ++i) {
            double t = Z[r * n + i];
            for (int k = 0; k < i; ++k) t -= L0[i * n + k] * Y[r * n + k];
            Y[r * n + i] = t / L0[i * n + i];
        }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) Y[i * n + j] = Y[j * n + i] = 0.5 * (Y[i * n + j] + Y[j * n + i]);
    std::vector<double> mu, E;
    sym_eigen(Y, n, mu, E);
    // Y is relative to X0: eigenvalues below 1e-9 in magnitude are rounding (kappa = 0: none)
    int npos = 0, nneg = 0;
    for (double m : mu) {
        npos += m > 1e-9;
        nneg += m < -1e-9;
    }
    if (npos > 1 || nneg > 1) return false;
    const double mp = mu[n - 1] > 1e-9 ? mu[n - 1] : 0.0, mm = mu[0] < -1e-9 ? mu[0] : 0.0;
    if (1.0 - S * (-mm) < -1e-9) return false;
    auto vec = [&](int col, double scl, double out[7]) {
        double vmax = 0.0;
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int k = 0; k <= i; ++k) t += L0[i * n + k] * E[k * n + col];
            out[i] = scl * t;
            vmax = std::max(vmax, std::fabs(out[i]));
        }
        for (int i = 0; i < n; ++i)
            if (std::fabs(out[i]) >= 0.5 * vmax) {
                if (out[i] < 0)
                    for (int k = 0; k < n; ++k) out[k] = -out[k];
                break;
            }
    };
    vec(n - 1, std::sqrt(mp), p);
    vec(0, std::sqrt(-mm), q);
    std::vector<double> C((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) C[i * n + j] = X0[i * n + j] - S * q[i] * q[j];
    return cholesky_block(C.data(), n, all, Lw);
}

// ---- populations in and out; sums ---------------------------------------------------------

// The stored geometry of a context (the padded storage of lb3d_kernel.cuh).
struct Geom3 {
    int nx, ny, nz, gx, pitch;
    long long PL, P;
    // stored offset of node (x, y, z), -gx <= x < nx + gx, -GY3 <= y < ny + GY3
    __host__ __device__ long long at(int x, int y, int z) const {
        return (long long)z * PL + (long long)(y + GY3) * pitch + (x + gx);
    }
};

// coordinates of lattice node q = (z ny + y) nx + x
__device__ __forceinline__ void coords3(long long q, int nx, int ny, int* x, int* y, int* z) {
    const long long nxy = (long long)nx * ny;
    *z = (int)(q / nxy);
    const long long r = q - (long long)*z * nxy;
    *y = (int)(r / nx);
    *x = (int)(r - (long long)*y * nx);
}

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// The device holds post-collision deviations (the kernel pulls f_i(r) = f*_i(r - c_i)), so
// the pre-collision f_i(r) of the ABI is stored at r - c_i: stored(q) = f_i(q + c_i) - fbar_i
// on the interior; fill_ghosts3_kernel then sets the ghost copies.
template <typename R>
__global__ void set_plane3_kernel(const double* __restrict__ src, R* __restrict__ dst, Geom3 g, int cx, int cy,
                                  int cz, double fbar) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords3(q, g.nx, g.ny, &x, &y, &z);
        const int sx = wrap1(x + cx, g.nx), sy = wrap1(y + cy, g.ny), sz = wrap1(z + cz, g.nz);
        dst[g.at(x, y, z)] = (R)(src[((long long)sz * g.ny + sy) * g.nx + sx] - fbar);
    }
}

// every ghost position of one population takes the value of the interior node it wraps to
template <typename R>
__global__ void fill_ghosts3_kernel(R* __restrict__ p, Geom3 g) {
    const int W = g.nx + 2 * g.gx, H = g.ny + 2 * GY3;
    const long long n = (long long)W * H * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(q / ((long long)W * H));
        const long long r = q - (long long)z * W * H;
        const int yy = (int)(r / W) - GY3, xx = (int)(r % W) - g.gx;
        if (xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny) continue;
        const int sx = ((xx % g.nx) + g.nx) % g.nx, sy = ((yy % g.ny) + g.ny) % g.ny;
        p[g.at(xx, yy, z)] = p[g.at(sx, sy, z)];
    }
}

// f_i(r) = stored(r - c_i) + fbar_i
template <typename R>
__global__ void get_plane3_kernel(const R* __restrict__ src, double* __restrict__ dst, Geom3 g, int cx, int cy,
                                  int cz, double fbar) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords3(q, g.nx, g.ny, &x, &y, &z);
        dst[q] = (double)src[g.at(wrap1(x - cx, g.nx), wrap1(y - cy, g.ny), wrap1(z - cz, g.nz))] + fbar;
    }
}

// adds delta to every stored element of one population (interior, ghosts and padding alike):
// the re-basing of the stored deviations on a new rest state
template <typename R>
__global__ void shift_plane3_kernel(R* __restrict__ p, long long n, double delta) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        p[q] = (R)((double)p[q] + delta);
}

// per-block FP64 partial sums of the density and momentum deviations over the interior
template <typename LAT, typename R>
__global__ void sums3_kernel(const R* __restrict__ p, Geom3 g, double* __restrict__ partial) {
    double s[4] = {0, 0, 0, 0};
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords3(k, g.nx, g.ny, &x, &y, &z);
        const long long o = g.at(x, y, z);
#pragma unroll
        for (int i = 0; i < LAT::Q; ++i) {
            const double f = (double)p[LAT::sigma(i) * g.P + o];
            s[0] += f;
            s[1] += LAT::c(i, 0) * f;
            s[2] += LAT::c(i, 1) * f;
            s[3] += LAT::c(i, 2) * f;
        }
    }
    __shared__ double red[4][256];
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) partial[blockIdx.x * 4 + q] = red[q][0];
}

constexpr int SUM3_BLOCKS = 256;

}  // namespace lbf3

using namespace lbf3;

struct lb3_ctx {
    int nx = 0, ny = 0, nz = 0, lattice = 19, precision = 0, device = 0, es = 4;
    long long n = 0;                // lattice nodes
    Geom3 geom{};                   // padded storage
    uint64_t seed = 0;
    double rho0 = 1.0;
    double cs2 = 1.0 / 3.0;         // c_s^2 of the linear theory about rho0
    double cs2_linear = 1.0 / 3.0;  // the cs2 of lb3_create (p0 = cs2 rho)
    int eos = LB_EOS_LINEAR;
    double eos_poly[5] = {};        // p0(rho0 + d) = sum_j eos_poly[j] d^j
    double eos_cq[4] = {};          // c_s^2(rho0 + d) = sum_j eos_cq[j] d^j
    double fbar[QMAX] = {};
    char* ws = nullptr;
    void* pop[2] = {nullptr, nullptr};
    double* stage = nullptr;        // one FP64 plane
    double* partial = nullptr;      // SUM3_BLOCKS x 4
    int* err_dev = nullptr;         // device error word of the TMA waits
    CUtensorMap maps[2][2];         // TMA: per configuration, the population buffers (box of its tile)
    int cur = 0;
    bool have_params = false;
    int noise_mode = LB_NOISE_OFF;
    double kT = 0, kappa = 0, tau_s = 1, tau_b = 1, tau_g = 1;
    Step3Args<float> af{};
    Step3Args<double> ad{};
    Launch3 cfg[2];                 // step kernel without / with the correlated noise (kmode 3)
    cudaStream_t stream = nullptr;
    long long t = 0;
    std::string err;
    int timing = 0;
    long long timing_seq = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t ev_used = 0;
    double ms_acc = 0.0;
    long long launches_acc = 0;
    long long kernels = 0;
};

namespace {
thread_local std::string g3_error;

int fail3(lb3_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg; else g3_error = msg;
    return code;
}

int cuda_fail3(lb3_ctx* c, cudaError_t e, const char* where) {
    return fail3(c, LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool sizes_ok(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return false;
    return (long double)nx * ny * nz < 4294967296.0L;
}

int es_of(int precision) { return precision == LB_FP32 ? 4 : (precision == LB_FP64 ? 8 : 0); }
bool lattice_ok(int lattice) { return lattice == LB_D3Q19 || lattice == LB_D3Q27; }

// padded storage of an nx x ny x nz lattice with es-byte elements (lb3d_kernel.cuh)
Geom3 geom3(int nx, int ny, int nz, int es) {
    Geom3 g{};
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.gx = 32 / es;
    g.pitch = ((nx + 2 * g.gx + g.gx - 1) / g.gx) * g.gx;
    g.PL = (long long)(ny + 2 * GY3) * g.pitch;
    g.P = (long long)nz * g.PL;
    return g;
}

struct Layout3 {
    size_t pop[2], stage, partial, err, total;
};

Layout3 layout3(const Geom3& g, int q, int es) {
    Layout3 L{};
    size_t off = 0;
    for (int k = 0; k < 2; ++k) {
        L.pop[k] = off;
        off = align256(off + (size_t)q * g.P * es);
    }
    L.stage = off;
    off = align256(off + (size_t)g.nx * g.ny * g.nz * sizeof(double));
    L.partial = off;
    off = align256(off + (size_t)SUM3_BLOCKS * 4 * sizeof(double));
    L.err = off;
    off = align256(off + sizeof(int));
    L.total = off;
    return L;
}

int record_timing3(lb3_ctx* c, cudaEvent_t* start, cudaEvent_t* stop) {
    if (c->ev_used == c->ev.size()) {
        if (c->ev.size() >= 1024) {
            cudaError_t e = cudaEventSynchronize(c->ev.back().second);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventSynchronize");
            for (auto& p : c->ev) {
                float ms = 0.f;
                e = cudaEventElapsedTime(&ms, p.first, p.second);
                if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventElapsedTime");
                c->ms_acc += ms;
            }
            c->ev_used = 0;
        } else {
            cudaEvent_t a, b;
            cudaError_t e = cudaEventCreate(&a);
            if (e == cudaSuccess) e = cudaEventCreate(&b);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventCreate");
            c->ev.push_back({a, b});
        }
    }
    *start = c->ev[c->ev_used].first;
    *stop = c->ev[c->ev_used].second;
    c->ev_used++;
    return LB_OK;
}

// The step kernel of a context.  Measured on GB300 at 256^3 (FP32): both lattices stage by
// TMA in two slots (D3Q19 without the correlated noise on 32 x 6 tiles, four CTAs per SM at
// 80 registers: 620 against 635 us on 32 x 8 and 681 us with three slots; with it on 32 x 8,
// 956 against 989 us on 32 x 6; D3Q27 on 32 x 4 tiles).  FP64 stages by copies
// (D3Q19 in three slots, D3Q27 in two; TMA boxes of doubles would fit one CTA per SM).
// LBFLUCT3_KERNEL=plain (D3Q19), LBFLUCT3_STAGE=tma|copy and LBFLUCT3_SLOTS=2|3 override
// the choice (32 x 6 tiles for D3Q27 by TMA measured 1063 against 1007 us: three CTAs per SM
// at 96 registers with spills).
Launch3 default_cfg(int lattice, int precision, bool rs) {
    Launch3 L{};
    L.kmode = 0;
    L.plain = false;
    L.tma = precision == LB_FP32;
    L.slots = (L.tma || lattice == 27) ? 2 : 3;
    L.ty = lattice == 19 ? ((L.tma && !rs) ? 6 : 8) : 4;
    return L;
}

Launch3 env_cfg(Launch3 L, int lattice, int precision, bool rs) {
    const char* v = std::getenv("LBFLUCT3_KERNEL");
    L.plain = v && std::strcmp(v, "plain") == 0 && lattice == 19 && !rs;
    if (const char* st = std::getenv("LBFLUCT3_STAGE")) {
        if (std::strcmp(st, "tma") == 0) L.tma = precision == LB_FP32;
        else if (std::strcmp(st, "copy") == 0) L.tma = false;
    }
    if (const char* sv = std::getenv("LBFLUCT3_SLOTS")) L.slots = std::atoi(sv) == 2 ? 2 : 3;
    if (lattice == 27 && L.tma) L.slots = 2;
    if (lattice == 19) L.ty = (L.tma && !rs) ? 6 : 8;      // the tiles the kernels are built for
    return L;
}

// The grid of a configuration: the z runs of the CTAs are at most RUN3 planes long, and short
// enough that there are CTAs for eight per SM.  Long runs let the CTAs of neighbouring tiles
// drift apart in z, so the halo one of them loads has left L2 before the other needs it:
// measured at 256^3 (FP32, TMA staging), 52-plane runs read 1.41x the algorithmic bytes and
// 16-plane runs 1.18x (D3Q19 657 -> 628 us, D3Q27 993 -> 859 us); 8-, 32- and 64-plane runs
// were slower.
constexpr int RUN3 = 16;

void choose_grid(lb3_ctx* c, Launch3* L) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int tx = 32, ty = L->plain ? 8 : L->ty;
    const long long bxy = (long long)((c->nx + tx - 1) / tx) * ((c->ny + ty - 1) / ty);
    const long long want = 8LL * sms;
    long long chunks = std::max((want + bxy - 1) / bxy, ((long long)c->nz + RUN3 - 1) / RUN3);
    chunks = std::max(1LL, std::min((long long)c->nz, chunks));
    const int zc = (int)((c->nz + chunks - 1) / chunks);
    chunks = (c->nz + zc - 1) / zc;
    L->grid = dim3((c->nx + tx - 1) / tx, (c->ny + ty - 1) / ty, (unsigned)chunks);
    L->zc = zc;
}

// Tensor map over one population buffer: dims (pitch, ny + 2 GY3, nz, Q) of FP32, box
// (TX + 8, ty + 2, 1, GM) (the tile, its ring and the 16-byte x alignment; the GM stored
// planes of one (c_y, c_z)), zero fill outside.
bool make_map3(const lb3_ctx* c, const void* buf, int ty, CUtensorMap* map) {
    lbf::EncodeTiledFn fn = lbf::tensor_map_encoder();
    if (!fn) return false;
    const Geom3& g = c->geom;
    cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * GY3), (cuuint64_t)g.nz,
                          (cuuint64_t)c->lattice};
    cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.PL * 4, (cuuint64_t)g.P * 4};
    cuuint32_t box[4] = {32 + 8, (cuuint32_t)(ty + 2), 1, (cuuint32_t)(c->lattice == 19 ? Lat19::GM : Lat27::GM)};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(buf), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Reads the device error word (after the stream has drained); a CTA that gave up waiting for
// its TMA loads is reported as LB_ETIMEOUT and the word cleared.
int check_device_error3(lb3_ctx* c) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "error word");
    if (h != 0) {
        e = cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return cuda_fail3(c, e, "error word");
        return fail3(c, LB_ETIMEOUT, "a 3-D step kernel gave up waiting for its TMA loads");
    }
    return LB_OK;
}

// Xi(0) of the lattice, row-major Q x Q
void xi_zero(int lattice, double rho0, double cs2, double kT, double tau_s, double tau_b, double tau_g, double* X) {
    if (lattice == 19) xi_zero19(rho0, cs2, kT, -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_g, X);
    else xi_zero27(rho0, cs2, kT, -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_g, X);
}

// noise factors of the kernel: sc = sqrt of the diagonal for the uncoupled modes, Lc the
// coupled block's Cholesky factor; false if Xi(0) is not positive semidefinite
bool noise_factors(int lattice, const double* X, double sc[QMAX], double Lc[28]) {
    const int Q = lattice;
    for (int k = 0; k < QMAX; ++k) sc[k] = 0.0;
    for (int k = 0; k < 28; ++k) Lc[k] = 0.0;
    const std::vector<int> coupled = lattice == 19 ? std::vector<int>{4, 16}
                                                   : std::vector<int>(COUPLED27, COUPLED27 + 7);
    std::vector<double> L;
    if (!cholesky_block(X, Q, coupled, L)) return false;
    const int n = (int)coupled.size();
    if (lattice == 19) {
        Lc[0] = L[0];
        Lc[1] = L[1 * n + 0];
        Lc[2] = L[1 * n + 1];
    } else {
        for (int r = 0; r < n; ++r)
            for (int q = 0; q <= r; ++q) Lc[r * (r + 1) / 2 + q] = L[r * n + q];
    }
    double scale = 1e-300;
    for (int k = 0; k < Q; ++k) scale = std::max(scale, std::fabs(X[k * Q + k]));
    for (int k = 0; k < Q; ++k) {
        if (std::find(coupled.begin(), coupled.end(), k) != coupled.end()) continue;
        const double v = X[k * Q + k];
        if (v < -1e-9 * scale) return false;
        sc[k] = std::sqrt(std::max(v, 0.0));
    }
    return true;
}

template <typename R>
void fill_args(lb3_ctx* c, Step3Args<R>* a, double tau_s, double tau_b, double tau_g, const double sc[QMAX],
               const double Lc[28], const double Lb[28], const double Lrs[12], const double Prs[7], const double Qrs[7]) {
    a->nx = c->nx; a->ny = c->ny; a->nz = c->nz;
    a->pitch = c->geom.pitch; a->gx = c->geom.gx; a->PL = c->geom.PL; a->P = c->geom.P;
    a->err = c->err_dev;
    a->co.rho0 = (R)c->rho0;
    a->co.d = (R)(3.0 * c->cs2 - 1.0);
    a->co.kappa = (R)c->kappa;
    a->co.lb = (R)(-1.0 / tau_b);
    a->co.ls = (R)(-1.0 / tau_s);
    a->co.lg = (R)(-1.0 / tau_g);
    a->co.e2 = (R)c->eos_poly[2];
    a->co.e3 = (R)c->eos_poly[3];
    a->co.e4 = (R)c->eos_poly[4];
    for (int q = 0; q < 4; ++q) a->cq[q] = (R)c->eos_cq[q];
    for (int q = 0; q < QMAX; ++q) a->sc[q] = (R)sc[q];
    for (int q = 0; q < 28; ++q) a->Lc[q] = (R)Lc[q];
    for (int q = 0; q < 28; ++q) a->Lb[q] = (R)Lb[q];
    for (int q = 0; q < 12; ++q) a->Lrs[q] = (R)Lrs[q];
    for (int q = 0; q < 7; ++q) {
        a->Prs[q] = (R)Prs[q];
        a->Qrs[q] = (R)Qrs[q];
    }
    a->rk = lbf::make_round_keys(c->seed);
}

template <typename R>
cudaError_t launch_any(lb3_ctx* c, Step3Args<R> a, int kmode) {
    const int q = kmode == 3 ? 1 : 0;
    Launch3 L = c->cfg[q];
    L.kmode = kmode;
    if (kmode == 4) L.plain = false;      // the plain kernel draws no local noise
    a.zc = L.zc;
    const CUtensorMap* map = &c->maps[q][c->cur];
    return c->lattice == 19 ? launch_lattice<Lat19, R>(a, map, L, c->stream)
                            : launch_lattice<Lat27, R>(a, map, L, c->stream);
}

}  // namespace

extern "C" {

size_t lb3_workspace_bytes(int nx, int ny, int nz, int lattice, int precision) {
    const int es = es_of(precision);
    if (!es || !lattice_ok(lattice) || !sizes_ok(nx, ny, nz)) return 0;
    return layout3(geom3(nx, ny, nz, es), lattice, es).total;
}

int lb3_create(int nx, int ny, int nz, int lattice, int precision, uint64_t seed, double rho0, double cs2,
               lb3_ctx** out) {
    if (!out) return fail3(nullptr, LB_EINVAL, "out is NULL");
    *out = nullptr;
    const int es = es_of(precision);
    if (!lattice_ok(lattice)) return fail3(nullptr, LB_EINVAL, "lattice must be LB_D3Q19 or LB_D3Q27");
    if (!es) return fail3(nullptr, LB_EINVAL, "precision must be LB_FP32 or LB_FP64");
    if (!sizes_ok(nx, ny, nz)) return fail3(nullptr, LB_EINVAL, "sizes must be >= 1 with nx*ny*nz < 2^32");
    if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail3(nullptr, LB_EINVAL, "rho0 must be positive");
    if (!(cs2 > 0.0) || !std::isfinite(cs2)) return fail3(nullptr, LB_EINVAL, "cs2 must be positive");
    lb3_ctx* c = new lb3_ctx();
    c->nx = nx; c->ny = ny; c->nz = nz; c->n = (long long)nx * ny * nz; c->lattice = lattice;
    c->precision = precision; c->es = es; c->seed = seed; c->rho0 = rho0; c->cs2 = cs2;
    c->cs2_linear = cs2;
    c->eos_poly[0] = cs2 * rho0;
    c->eos_poly[1] = cs2;
    c->eos_cq[0] = cs2;
    cudaGetDevice(&c->device);
    c->geom = geom3(nx, ny, nz, es);
    const Layout3 L = layout3(c->geom, lattice, es);
    cudaError_t e = cudaMalloc((void**)&c->ws, L.total);
    if (e != cudaSuccess) {
        delete c;
        return fail3(nullptr, LB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->pop[0] = c->ws + L.pop[0];
    c->pop[1] = c->ws + L.pop[1];
    c->stage = (double*)(c->ws + L.stage);
    c->partial = (double*)(c->ws + L.partial);
    c->err_dev = (int*)(c->ws + L.err);
    rest_pops(lattice, rho0, cs2 * rho0, c->fbar);
    // the whole workspace starts at zero: the rest state, ghosts included
    e = cudaMemset(c->ws, 0, L.total);
    if (e != cudaSuccess) {
        cudaFree(c->ws);
        delete c;
        return fail3(nullptr, LB_ECUDA, std::string("lb3_create: ") + cudaGetErrorString(e));
    }
    std::memset(c->maps, 0, sizeof(c->maps));
    for (int k = 0; k < 2; ++k) {
        c->cfg[k] = env_cfg(default_cfg(lattice, precision, k == 1), lattice, precision, k == 1);
        choose_grid(c, &c->cfg[k]);
    }
    // a tensor-map pair per configuration that stages by TMA (its tile height sets the box)
    for (int q = 0; q < 2; ++q) {
        if (!c->cfg[q].tma) continue;
        for (int k = 0; k < 2; ++k)
            if (!make_map3(c, c->pop[k], c->cfg[q].ty, &c->maps[q][k])) {
                cudaFree(c->ws);
                delete c;
                return fail3(nullptr, LB_ECUDA, "lb3_create: cuTensorMapEncodeTiled failed");
            }
    }
    *out = c;
    return LB_OK;
}

int lb3_destroy(lb3_ctx* c) {
    if (!c) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (auto& p : c->ev) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    cudaFree(c->ws);
    delete c;
    return LB_OK;
}

int lb3_set_stream(lb3_ctx* c, void* stream) {
    if (!c) return LB_EINVAL;
    c->stream = (cudaStream_t)stream;
    return LB_OK;
}

int lb3_noise_matrix(int lattice, double rho0, double cs2, double kT, double tau_s, double tau_b, double tau_ghost,
                     double* xi) {
    if (!xi || !lattice_ok(lattice) || !(rho0 > 0) || !(cs2 > 0) || kT < 0 || !(tau_s > 0.5) || !(tau_b > 0.5) ||
        !(tau_ghost > 0.5))
        return LB_EINVAL;
    xi_zero(lattice, rho0, cs2, kT, tau_s, tau_b, tau_ghost, xi);
    return LB_OK;
}

int lb3_set_params(lb3_ctx* c, double kT, double kappa, double tau_s, double tau_b, double tau_ghost, int mode) {
    if (!c) return LB_EINVAL;
    if (!(tau_s > 0.5) || !(tau_b > 0.5) || !(tau_ghost > 0.5) || !std::isfinite(tau_s) || !std::isfinite(tau_b) ||
        !std::isfinite(tau_ghost))
        return fail3(c, LB_EINVAL, "relaxation times must exceed 1/2");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return fail3(c, LB_EINVAL, "kT must be >= 0");
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) return fail3(c, LB_EINVAL, "kappa must be >= 0");
    if (mode != LB_NOISE_OFF && mode != LB_NOISE_LW && mode != LB_NOISE_LW_LOCAL && mode != LB_NOISE_FULL_RS)
        return fail3(c, LB_EINVAL,
                     "the 3-D lattices take LB_NOISE_OFF, LB_NOISE_LW, LB_NOISE_FULL_RS or LB_NOISE_LW_LOCAL");
    const bool homogeneous = mode == LB_NOISE_LW || mode == LB_NOISE_FULL_RS;
    if (homogeneous && kT > 0 && !(c->cs2 > 0.0))
        return fail3(c, LB_ENOTPSD, "the linear theory about rho0 has c_s^2 <= 0 (a mean density in the spinodal region)");
    std::vector<double> X((size_t)c->lattice * c->lattice);
    double sc[QMAX] = {}, Lc[28] = {}, Lb[28] = {}, Lrs[12] = {}, Prs[7] = {}, Qrs[7] = {};
    if (homogeneous && kT > 0) {
        xi_zero(c->lattice, c->rho0, c->cs2, kT, tau_s, tau_b, tau_ghost, X.data());
        if (!noise_factors(c->lattice, X.data(), sc, Lc)) return fail3(c, LB_ENOTPSD, "Xi(0) is not positive semidefinite");
    }
    if (mode == LB_NOISE_LW_LOCAL && kT > 0) {
        // Xi(0) of a homogeneous system at density rho and sound speed c_s^2 is rho (A + B c_s^2)
        // entrywise (affine in c_s^2, linear in rho): A and B from two evaluations at rho = 1;
        // the kernel factors the coupled block at every node, the other modes scale with
        // sqrt(rho) (their B is zero)
        const int Q = c->lattice;
        const double c1 = 0.2, c2 = 0.4;
        std::vector<double> X2((size_t)Q * Q);
        xi_zero(Q, 1.0, c1, kT, tau_s, tau_b, tau_ghost, X.data());
        xi_zero(Q, 1.0, c2, kT, tau_s, tau_b, tau_ghost, X2.data());
        auto B = [&](int i, int j) { return (X2[i * Q + j] - X[i * Q + j]) / (c2 - c1); };
        auto A = [&](int i, int j) { return X[i * Q + j] - c1 * B(i, j); };
        std::vector<int> coupled = Q == 19 ? std::vector<int>{4, 16} : std::vector<int>(COUPLED27, COUPLED27 + 7);
        for (int k = 0; k < Q; ++k) {
            if (std::find(coupled.begin(), coupled.end(), k) != coupled.end()) continue;
            sc[k] = std::sqrt(std::max(A(k, k), 0.0));
        }
        const int n = (int)coupled.size();
        for (int r = 0; r < n; ++r)
            for (int q = 0; q <= r; ++q) {
                Lc[r * (r + 1) / 2 + q] = A(coupled[r], coupled[q]);
                Lb[r * (r + 1) / 2 + q] = B(coupled[r], coupled[q]);
            }
    }
    if (mode == LB_NOISE_FULL_RS && kT > 0 && c->lattice == 27) {
        // Xi(k) is Xi(0) at c_s^2(k) = cs2 + rho0 kappa s(k), s = 6 (1 - prod (2 + cos k_a) / 3)
        // (multilinear in the cosines, corner values 0, 4, 16/3, 52/9): the rank-two split of
        // its coupled block; the white part's factor replaces Xi(0)'s in Lc, and the fields
        // along p and q take the corner amplitudes sqrt(s) and sqrt(52/9 - s)
        const double svals[4] = {0.0, 4.0, 16.0 / 3.0, 52.0 / 9.0};
        std::vector<double> Lw;
        if (!rs_split27(c->rho0, c->cs2, kappa, kT, -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_ghost, Lw, Prs, Qrs))
            return fail3(c, LB_ENOTPSD, "Xi(k) is not positive semidefinite on the lattice");
        for (int r = 0; r < 7; ++r)
            for (int p2 = 0; p2 <= r; ++p2) Lc[r * (r + 1) / 2 + p2] = Lw[r * 7 + p2];
        for (int q = 0; q < 4; ++q) {
            Lrs[3 * q] = std::sqrt(svals[q]);
            Lrs[3 * q + 1] = 0.0;
            Lrs[3 * q + 2] = std::sqrt(std::max(svals[3] - svals[q], 0.0));
        }
    }
    if (mode == LB_NOISE_FULL_RS && kT > 0 && c->lattice == 19) {
        // Xi(k) is Xi(0) at c_s^2(k) = cs2 + rho0 kappa s(k); the factors of its (4,16) block at
        // the corner values s = 0, 4, 16/3 (positive semidefinite there means at every k)
        const double svals[3] = {0.0, 4.0, 16.0 / 3.0};
        for (int q = 0; q < 3; ++q) {
            std::vector<double> Xs((size_t)Q3 * Q3);
            xi_zero19(c->rho0, c->cs2 + c->rho0 * kappa * svals[q], kT, -1.0 / tau_b, -1.0 / tau_s,
                      -1.0 / tau_ghost, Xs.data());
            std::vector<double> L2;
            if (!cholesky_block(Xs.data(), Q3, {4, 16}, L2))
                return fail3(c, LB_ENOTPSD, "Xi(k) is not positive semidefinite on the lattice");
            Lrs[3 * q] = L2[0];
            Lrs[3 * q + 1] = L2[2];
            Lrs[3 * q + 2] = L2[3];
        }
    }
    c->kT = kT;
    c->kappa = kappa;
    c->tau_s = tau_s; c->tau_b = tau_b; c->tau_g = tau_ghost;
    c->noise_mode = mode;
    fill_args(c, &c->af, tau_s, tau_b, tau_ghost, sc, Lc, Lb, Lrs, Prs, Qrs);
    fill_args(c, &c->ad, tau_s, tau_b, tau_ghost, sc, Lc, Lb, Lrs, Prs, Qrs);
    c->have_params = true;
    return LB_OK;
}

static unsigned plane_blocks(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 4096); }

int lb3_set_eos(lb3_ctx* c, int eos, double beta, double rhoV, double rhoL) {
    if (!c) return LB_EINVAL;
    if (eos != LB_EOS_LINEAR && eos != LB_EOS_DOUBLE_WELL) return fail3(c, LB_EINVAL, "unknown equation of state");
    const double r0 = c->rho0;
    double poly[5] = {0, 0, 0, 0, 0}, cq[4] = {0, 0, 0, 0};
    if (eos == LB_EOS_DOUBLE_WELL) {
        if (!(beta > 0.0) || !std::isfinite(beta) || !(rhoV >= 0.0) || !(rhoL > rhoV) || !std::isfinite(rhoL))
            return fail3(c, LB_EINVAL, "the double well needs beta > 0 and 0 <= rhoV < rhoL");
        // f0(rho0 + d) / beta = (A + d)^2 (B + d)^2 with A = rho0 - rhoV, B = rho0 - rhoL, as a
        // polynomial in d; p0 = rho df0/drho - f0 and c_s^2 = rho d2f0/drho2 in the same form
        const double A = r0 - rhoV, B = r0 - rhoL, s0 = A * B, s1 = A + B;
        const double f[5] = {s0 * s0, 2 * s0 * s1, s1 * s1 + 2 * s0, 2 * s1, 1.0};
        double df[4], d2f[3];
        for (int j = 0; j < 4; ++j) df[j] = (j + 1) * f[j + 1];
        for (int j = 0; j < 3; ++j) d2f[j] = (j + 1) * df[j + 1];
        for (int j = 0; j < 5; ++j) poly[j] = beta * ((j < 4 ? r0 * df[j] : 0.0) + (j >= 1 ? df[j - 1] : 0.0) - f[j]);
        for (int j = 0; j < 4; ++j) cq[j] = beta * ((j < 3 ? r0 * d2f[j] : 0.0) + (j >= 1 ? d2f[j - 1] : 0.0));
    } else {
        poly[0] = c->cs2_linear * r0;
        poly[1] = c->cs2_linear;
        cq[0] = c->cs2_linear;
    }
    lbf::DeviceGuard dg(c->device);
    // the stored deviations, re-based on the rest state of the new equation of state
    double fb_new[QMAX] = {};
    rest_pops(c->lattice, r0, poly[0], fb_new);
    const long long P = c->geom.P;
    for (int i = 0; i < c->lattice; ++i) {
        const long long off = (long long)sigma_of(c->lattice, i) * P;
        const double delta = c->fbar[i] - fb_new[i];
        if (c->precision == LB_FP64)
            shift_plane3_kernel<double><<<plane_blocks(P), 256, 0, c->stream>>>((double*)c->pop[c->cur] + off, P, delta);
        else
            shift_plane3_kernel<float><<<plane_blocks(P), 256, 0, c->stream>>>((float*)c->pop[c->cur] + off, P, delta);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail3(c, e, "re-base populations");
        c->kernels += 1;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    for (int i = 0; i < c->lattice; ++i) c->fbar[i] = fb_new[i];
    c->eos = eos;
    for (int j = 0; j < 5; ++j) c->eos_poly[j] = poly[j];
    for (int j = 0; j < 4; ++j) c->eos_cq[j] = cq[j];
    c->cs2 = poly[1];                     // c_s^2 of the linear theory about rho0
    if (c->have_params) {
        const int r = lb3_set_params(c, c->kT, c->kappa, c->tau_s, c->tau_b, c->tau_g, c->noise_mode);
        if (r != LB_OK) {
            c->have_params = false;        // the old noise factors belong to the old equation of state
            return r;
        }
    }
    return LB_OK;
}

int lb3_step(lb3_ctx* c, int64_t nsteps) {
    if (!c) return LB_EINVAL;
    if (nsteps < 0) return fail3(c, LB_EINVAL, "nsteps must be >= 0");
    if (!c->have_params) return fail3(c, LB_ESTATE, "lb3_set_params must be called before lb3_step");
    lbf::DeviceGuard dg(c->device);
    const int kmode = c->kT > 0.0 ? (c->noise_mode == LB_NOISE_LW ? 1
                                     : (c->noise_mode == LB_NOISE_FULL_RS ? 3
                                        : (c->noise_mode == LB_NOISE_LW_LOCAL ? 4 : 0)))
                                  : 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        const uint32_t tlo = (uint32_t)((uint64_t)c->t & 0xffffffffu), thi = (uint32_t)((uint64_t)c->t >> 32);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        const bool tm = c->timing > 0 && (c->timing_seq++ % c->timing) == 0;
        if (tm) {
            int r = record_timing3(c, &e0, &e1);
            if (r != LB_OK) return r;
            cudaError_t e = cudaEventRecord(e0, c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventRecord");
        }
        cudaError_t e;
        if (c->precision == LB_FP64) {
            Step3Args<double> a = c->ad;
            a.src = (const double*)c->pop[c->cur];
            a.dst = (double*)c->pop[c->cur ^ 1];
            a.t_lo = tlo; a.t_hi = thi;
            e = launch_any(c, a, kmode);
        } else {
            Step3Args<float> a = c->af;
            a.src = (const float*)c->pop[c->cur];
            a.dst = (float*)c->pop[c->cur ^ 1];
            a.t_lo = tlo; a.t_hi = thi;
            e = launch_any(c, a, kmode);
        }
        if (e != cudaSuccess) return cuda_fail3(c, e, "3-D step kernel launch");
        c->kernels += 1;
        if (tm) {
            e = cudaEventRecord(e1, c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventRecord");
            c->launches_acc++;
        }
        c->cur ^= 1;
        c->t++;
    }
    return LB_OK;
}

int lb3_get_time(lb3_ctx* c, int64_t* t) {
    if (!c || !t) return LB_EINVAL;
    *t = c->t;
    return LB_OK;
}


int lb3_set_populations(lb3_ctx* c, const double* f, int loc, int64_t t) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE) || t < 0) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (int i = 0; i < c->lattice; ++i) {
        const double* src = f + (long long)i * c->n;
        if (loc == LB_HOST) {
            cudaError_t e = cudaMemcpyAsync(c->stage, src, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "H2D");
            src = c->stage;
        }
        const int cx = c_of(c->lattice, i, 0), cy = c_of(c->lattice, i, 1), cz = c_of(c->lattice, i, 2);
        const Geom3& g = c->geom;
        const long long padded = (long long)(g.nx + 2 * g.gx) * (g.ny + 2 * GY3) * g.nz;
        if (c->precision == LB_FP64) {
            double* p = (double*)c->pop[c->cur] + (long long)sigma_of(c->lattice, i) * g.P;
            set_plane3_kernel<double><<<plane_blocks(c->n), 256, 0, c->stream>>>(src, p, g, cx, cy, cz, c->fbar[i]);
            fill_ghosts3_kernel<double><<<plane_blocks(padded), 256, 0, c->stream>>>(p, g);
        } else {
            float* p = (float*)c->pop[c->cur] + (long long)sigma_of(c->lattice, i) * g.P;
            set_plane3_kernel<float><<<plane_blocks(c->n), 256, 0, c->stream>>>(src, p, g, cx, cy, cz, c->fbar[i]);
            fill_ghosts3_kernel<float><<<plane_blocks(padded), 256, 0, c->stream>>>(p, g);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail3(c, e, "set populations");
        c->kernels += 2;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    c->t = t;
    return LB_OK;
}

int lb3_get_populations(lb3_ctx* c, double* f, int loc) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE)) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (int i = 0; i < c->lattice; ++i) {
        double* dst = loc == LB_HOST ? c->stage : f + (long long)i * c->n;
        const int cx = c_of(c->lattice, i, 0), cy = c_of(c->lattice, i, 1), cz = c_of(c->lattice, i, 2);
        const Geom3& g = c->geom;
        if (c->precision == LB_FP64)
            get_plane3_kernel<double><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                (const double*)c->pop[c->cur] + (long long)sigma_of(c->lattice, i) * g.P, dst, g, cx, cy, cz, c->fbar[i]);
        else
            get_plane3_kernel<float><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                (const float*)c->pop[c->cur] + (long long)sigma_of(c->lattice, i) * g.P, dst, g, cx, cy, cz, c->fbar[i]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail3(c, e, "get populations");
        c->kernels += 1;
        if (loc == LB_HOST) {
            e = cudaMemcpyAsync(f + (long long)i * c->n, c->stage, sizeof(double) * c->n, cudaMemcpyDeviceToHost,
                                c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "D2H");
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    return check_device_error3(c);
}

int lb3_sums(lb3_ctx* c, double sums[4]) {
    if (!c || !sums) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    const bool d = c->precision == LB_FP64;
    if (c->lattice == 19) {
        if (d)
            sums3_kernel<Lat19, double><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const double*)c->pop[c->cur], c->geom,
                                                                           c->partial);
        else
            sums3_kernel<Lat19, float><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const float*)c->pop[c->cur], c->geom,
                                                                          c->partial);
    } else {
        if (d)
            sums3_kernel<Lat27, double><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const double*)c->pop[c->cur], c->geom,
                                                                           c->partial);
        else
            sums3_kernel<Lat27, float><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const float*)c->pop[c->cur], c->geom,
                                                                          c->partial);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail3(c, e, "sums kernel");
    c->kernels += 1;
    std::vector<double> h((size_t)SUM3_BLOCKS * 4);
    e = cudaMemcpyAsync(h.data(), c->partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "sums D2H");
    if (int r = check_device_error3(c)) return r;
    double s[4] = {0, 0, 0, 0};
    for (int b = 0; b < SUM3_BLOCKS; ++b)
        for (int q = 0; q < 4; ++q) s[q] += h[(size_t)b * 4 + q];
    sums[0] = c->rho0 * (double)c->n + s[0];
    sums[1] = s[1];
    sums[2] = s[2];
    sums[3] = s[3];
    return LB_OK;
}

int lb3_set_kernel_timing(lb3_ctx* c, int every) {
    if (!c) return LB_EINVAL;
    if (every < 0) return fail3(c, LB_EINVAL, "timing stride must be >= 0");
    c->timing = every;
    c->timing_seq = 0;
    c->ev_used = 0;
    c->ms_acc = 0.0;
    c->launches_acc = 0;
    return LB_OK;
}

int lb3_kernel_time(lb3_ctx* c, double* ms, int64_t* launches) {
    if (!c) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    double total = c->ms_acc;
    if (c->ev_used > 0) {
        cudaError_t e = cudaEventSynchronize(c->ev[c->ev_used - 1].second);
        if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventSynchronize");
        for (size_t k = 0; k < c->ev_used; ++k) {
            float v = 0.f;
            e = cudaEventElapsedTime(&v, c->ev[k].first, c->ev[k].second);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventElapsedTime");
            total += v;
        }
    }
    if (ms) *ms = total;
    if (launches) *launches = c->launches_acc;
    return LB_OK;
}

int lb3_launch_count(lb3_ctx* c, int64_t* launches) {
    if (!c || !launches) return LB_EINVAL;
    *launches = c->kernels;
    return LB_OK;
}

int lb3_synchronize(lb3_ctx* c) {
    if (!c) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    return check_device_error3(c);
}

const char* lb3_last_error(lb3_ctx* c) { return c ? c->err.c_str() : g3_error.c_str(); }

}  // extern "C"
