// lb_api.cu -- the C ABI declared in include/lbfluct.h.
//
// Host side: context and workspace management, the FP64 parameter theory of
// [GACV] Sec. III C-IV (noise covariance Xi(k) of Eq. noise-yeo, its positive
// semidefiniteness on the lattice's wavevectors, the Cholesky factors of Sec. IV),
// and the launch sequence of one time step.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "lb_internal.cuh"
#include "lbfluct.h"

using namespace lbf;

namespace {

constexpr double SIGMA_S2 = 1.0 / 3.0;   // [GACV] Sec. III, notation
thread_local std::string g_create_error;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool is_pow2(int v) { return v >= 2 && (v & (v - 1)) == 0; }

struct WsLayout {
    size_t pop[2], z1, z2, twx, twy, cosx, cosy, bins, counts, bin16, partial, sums3, fbar, err, total;
    size_t twxd, twyd, cosxd, cosyd;   // FP64 storage: FP64 tables of the correlated noise
};

int elem_size(int precision) {
    return precision == LB_FP16DEV ? 2 : (precision == LB_FP32 ? 4 : (precision == LB_FP64 ? 8 : 0));
}

bool make_grid(int nx, int ny, int esize, Grid* g) {
    if (nx < 2 || ny < 2 || nx > (1 << 16) || ny > (1 << 16) || esize <= 0) return false;
    const int line = 128 / esize;                 // elements per 128 bytes
    g->nx = nx;
    g->ny = ny;
    g->gx = line;
    g->pitch = (nx + 2 * line + line - 1) / line * line;
    const long long a256 = 256 / esize;
    g->plane = ((long long)g->pitch * (ny + 2 * GY) + a256 - 1) / a256 * a256;
    return true;
}

WsLayout make_layout(const Grid& g, int esize) {
    WsLayout L{};
    const long long n = (long long)g.nx * g.ny;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L.pop[0] = take((size_t)Q * g.plane * esize);
    L.pop[1] = take((size_t)Q * g.plane * esize);
    // z1 holds the correlated noise (complex, FP64 with FP64 storage) and spectra scratch
    L.z1 = take((size_t)n * (esize == 8 ? sizeof(double2) : sizeof(float2)));
    L.z2 = take((size_t)n * sizeof(float2));
    L.twx = take((size_t)g.nx * sizeof(float2));
    L.twy = take((size_t)g.ny * sizeof(float2));
    L.cosx = take((size_t)g.nx * sizeof(float));
    L.cosy = take((size_t)g.ny * sizeof(float));
    L.bins = take((size_t)3 * MAX_BINS * sizeof(double));
    L.counts = take((size_t)MAX_BINS * sizeof(unsigned long long));
    L.bin16 = take((size_t)n * sizeof(unsigned short));
    L.partial = take((size_t)sums_partial_count() * sizeof(double));
    L.sums3 = take(3 * sizeof(double));
    L.fbar = take(Q * sizeof(double));
    L.err = take(sizeof(int));
    L.twxd = L.twyd = L.cosxd = L.cosyd = 0;
    if (esize == 8) {
        L.twxd = take((size_t)g.nx * sizeof(double2));
        L.twyd = take((size_t)g.ny * sizeof(double2));
        L.cosxd = take((size_t)g.nx * sizeof(double));
        L.cosyd = take((size_t)g.ny * sizeof(double));
    }
    L.total = off;
    return L;
}

// velocities in [GACV] Eq. (Tmat) order and the D2Q9 weights (Sec. III A)
const int CXh[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int CYh[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const double Wh[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

// Noise covariance of [GACV] Eq. (noise-yeo) as functions of the lattice k^2 (s):
// Xi_44 = a44 + b44 s, Xi_49 = a49 + b49 s, Xi_99 = a99 + b99 s; the shear and ghost
// entries do not depend on k.
struct NoiseCoef {
    double a44, b44, a49, b49, a99, b99, x55, x66, x77;
};

NoiseCoef noise_coef(double rho0, double cs2, double kT, double kappa, double tau_s, double tau_b,
                     double tau_g) {
    const double lb = -1.0 / tau_b, ls = -1.0 / tau_s, lq = -1.0 / tau_g, le = -1.0 / tau_g;
    const double til_b = lb * (2.0 + lb), til_s = ls * (2.0 + ls), til_q = lq * (2.0 + lq);
    const double til_e = le * (2.0 + le), til_be = lb + le + lb * le;
    const double pref = -(rho0 * kT / SIGMA_S2);
    const double N4 = 4.0, N5 = 4.0 / 9.0, N6 = 1.0 / 9.0, N7 = 2.0 / 3.0, N9 = 16.0;
    NoiseCoef c;
    // c_s^2(k) = cs2 + rho0 kappa s
    c.a44 = pref * N4 * (2.0 - 3.0 * cs2) * til_b;
    c.b44 = pref * N4 * (-3.0 * rho0 * kappa) * til_b;
    c.a49 = pref * 12.0 * (cs2 - SIGMA_S2) * til_be;
    c.b49 = pref * 12.0 * (rho0 * kappa) * til_be;
    c.a99 = pref * N9 * (1.25 - 0.75 * cs2) * til_e;
    c.b99 = pref * N9 * (-0.75 * rho0 * kappa) * til_e;
    c.x55 = pref * N5 * til_s;
    c.x66 = pref * N6 * til_s;
    c.x77 = pref * N7 * til_q;
    return c;
}

// largest lattice k^2 (at k = (pi, pi)), and the k^2 of the middle factor of the real-space
// correlated noise (LB_NOISE_FULL_RS, lb_internal.cuh stencil_h)
constexpr double S_MAX = 16.0 / 3.0;
constexpr double S_MID = 4.0;

// lattice k^2: minus the Fourier symbol of the Appendix B Laplacian
double k2_lattice(double kx, double ky) {
    return -((4.0 / 9.0) * (std::cos(kx) + std::cos(ky)) + (2.0 / 9.0) * std::cos(kx) * std::cos(ky) - 10.0 / 9.0) /
           SIGMA_S2;
}

bool block_psd(const NoiseCoef& c, double s) {
    const double x44 = c.a44 + c.b44 * s, x49 = c.a49 + c.b49 * s, x99 = c.a99 + c.b99 * s;
    const double scale = std::fmax(std::fabs(x44), std::fabs(x99)) + 1e-300;
    const double tol = 1e-12 * scale;
    if (x44 < -tol || x99 < -tol) return false;
    return x44 * x99 - x49 * x49 >= -tol * scale;
}

// Factor L = S diag(sqrt e1, sqrt e2) of the PSD block [[a, b], [b, c]] (Sec. IV, the
// eigen-decomposition alternative to Cholesky): e1 >= e2 its eigenvalues and
// S = [[cos t, -sin t], [sin t, cos t]], t in [0, pi) with tan 2t = 2b / (a - c).
void eigen_factor_2x2(double a, double b, double c, double* l11, double* l12, double* l21, double* l22) {
    const double half = 0.5 * (a + c);
    const double rad = std::sqrt(0.25 * (a - c) * (a - c) + b * b);
    const double e1 = half + rad, e2 = std::fmax(half - rad, 0.0);
    double t = 0.5 * std::atan2(2.0 * b, a - c);
    if (t < 0.0) t += M_PI;
    const double r1 = std::sqrt(std::fmax(e1, 0.0)), r2 = std::sqrt(e2);
    *l11 = std::cos(t) * r1;
    *l12 = -std::sin(t) * r2;
    *l21 = std::sin(t) * r1;
    *l22 = std::cos(t) * r2;
}

int validate(int nx, int ny, double rho0, double cs2, double kT, double kappa, double tau_s, double tau_b,
             double tau_g, int mode, std::string* why) {
    auto bad = [&](const char* m) { if (why) *why = m; return LB_EINVAL; };
    if (!(tau_s > 0.5) || !(tau_b > 0.5) || !(tau_g > 0.5)) return bad("every relaxation time must exceed 1/2");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return bad("kT must be finite and >= 0");
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) return bad("kappa must be finite and >= 0");
    if (mode < LB_NOISE_OFF || mode > LB_NOISE_LW_LOCAL) return bad("unknown noise mode");
    if (!(rho0 > 0.0)) return bad("rho0 must be positive");
    // the local-density noise factors Xi(0) per node (negative pivots clamped): no
    // homogeneous state to check
    if (mode == LB_NOISE_OFF || kT == 0.0 || mode == LB_NOISE_LW_LOCAL) return LB_OK;
    if (!(cs2 > 0.0)) return bad("the sound speed squared of the state about rho0 must be positive");
    const NoiseCoef c = noise_coef(rho0, cs2, 1.0, kappa, tau_s, tau_b, tau_g);
    if (mode == LB_NOISE_FULL) {
        // every wavevector of the lattice; cos is even, so the quarter grid suffices
        for (int my = 0; my <= ny / 2; ++my)
            for (int mx = 0; mx <= nx / 2; ++mx) {
                const double s = k2_lattice(2.0 * M_PI * mx / nx, 2.0 * M_PI * my / ny);
                if (!block_psd(c, s)) {
                    if (why) *why = "noise covariance Xi(k) is not positive semidefinite on this lattice";
                    return LB_ENOTPSD;
                }
            }
    } else if (mode == LB_NOISE_FULL_RS) {
        // Xi is affine in the lattice k^2 over [0, 16/3]: PSD at both ends <=> PSD for all k
        if (!block_psd(c, 0.0) || !block_psd(c, S_MAX)) {
            if (why) *why = "noise covariance Xi is not positive semidefinite at lattice k^2 = 0 or 16/3";
            return LB_ENOTPSD;
        }
    } else if (mode == LB_NOISE_LW) {
        if (!block_psd(c, 0.0)) {
            if (why) *why = "noise covariance Xi(0) is not positive semidefinite";
            return LB_ENOTPSD;
        }
    } else {   // LB_NOISE_DIAG uses the diagonal of Xi(0) only
        if (c.a44 < 0.0 || c.a99 < 0.0) {
            if (why) *why = "diagonal of Xi(0) has a negative entry";
            return LB_ENOTPSD;
        }
    }
    return LB_OK;
}

}  // namespace

struct lb_ctx {
    int nx = 0, ny = 0, precision = 0, device = 0, fp16 = 0;
    long long n = 0;
    uint64_t seed = 0;
    double rho0 = 1.0, cs2 = SIGMA_S2;
    Grid g{};
    WsLayout L{};
    char* ws = nullptr;
    bool owns = false;
    void* pop[2] = {nullptr, nullptr};
    int cur = 0;
    float2 *z1 = nullptr, *z2 = nullptr, *twx = nullptr, *twy = nullptr;
    float *cosx = nullptr, *cosy = nullptr;
    double *bins = nullptr, *partial = nullptr, *sums3 = nullptr, *fbar_dev = nullptr;
    unsigned long long* counts = nullptr;
    unsigned short* bin16 = nullptr;     // radial bin of every wavevector (spectra)
    int* err_dev = nullptr;          // set by a kernel whose bounded wait gave up
    bool pow2 = false;
    bool use_tma = false;            // TMA-staged persistent step kernel
    bool use_sweep = false;          // warp-autonomous vertical sweep kernel
    int sweep_occ6 = 0;              // its occupancy variant
    int tma_tile = 0;                // tile shape of the tensor maps (see lb_step_tma.cu)
    int tma_tile_fixed = -1;         // LBFLUCT_TMA_TILE, else -1: the fastest for the noise mode
    alignas(64) unsigned char tmap[2][128];
    double fbar[Q] = {};
    // parameters
    bool have_params = false;
    int noise_mode = LB_NOISE_OFF, warnings = 0;
    // equation of state (lb_set_eos): cs2 above is the sound speed squared of the linear
    // theory about rho0 (the lb_create argument for the linear EOS, c_s^2(rho0) for a double
    // well), p0_rest the bulk pressure of the rest state
    int eos = LB_EOS_LINEAR;
    double cs2_linear = 1.0 / 3.0, p0_rest = 1.0 / 3.0;
    double eos_beta = 0, eos_rhoV = 0, eos_rhoL = 0;
    double eos_poly[5] = {0, 0, 0, 0, 0};   // p0(rho0 + d) = sum_j eos_poly[j] d^j
    double eos_cq[4] = {0, 0, 0, 0};        // c_s^2(rho0 + d) = sum_j eos_cq[j] d^j
    int factor = LB_FACTOR_CHOLESKY;
    double kT = 0, kappa = 0, tau_s = 1, tau_b = 1, tau_g = 1;
    StepArgs sa{};
    NoiseGenArgs ga{};
    StepArgsD sad{};                 // FP64 storage
    NoiseGenArgsD gad{};
    double2 *twxd = nullptr, *twyd = nullptr;
    double *cosxd = nullptr, *cosyd = nullptr;
    // sampling
    int every = 0, nbins = 0;
    long long nsamples = 0;
    std::vector<unsigned long long> hcounts;
    // execution
    cudaStream_t stream = nullptr;
    long long t = 0;
    std::string err;
    // kernel timing
    int timing = 0;                 // 0 off, k: events around every k-th step-kernel launch
    long long timing_seq = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t ev_used = 0;
    double ms_acc = 0.0;
    long long launches_acc = 0;
    long long kernels = 0;          // every kernel launched on behalf of this context
};

namespace lbf {
void set_context_free_error(const std::string& msg) { g_create_error = msg; }

void noise_coefficients(double rho0, double cs2, double kT, double kappa, double tau_s, double tau_b,
                        double tau_ghost, double out[6]) {
    const NoiseCoef c = noise_coef(rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost);
    out[0] = c.a44; out[1] = c.b44; out[2] = c.a49; out[3] = c.b49; out[4] = c.a99; out[5] = c.b99;
}

// Rest populations fbar_i = w_i (rho0 + T_4i d rho0 / N_4 - T_9i d rho0 / N_9) for the
// reference moments {rho0, 0, 0, d rho0, 0, 0, 0, 0, -d rho0}, d = 6 (cs2 - sigma_s^2)
// (Table II at u = 0 with p0 = cs2 rho; inverse transform of Sec. III A).
void rest_populations(double rho0, double cs2, double fbar[Q]) {
    const double d = 6.0 * (cs2 - SIGMA_S2);
    for (int i = 0; i < Q; ++i) {
        const double c2 = CXh[i] * CXh[i] + CYh[i] * CYh[i];
        const double t4 = 3.0 * c2 - 2.0;
        const double t9 = 9.0 * c2 * c2 - 15.0 * c2 + 2.0;
        fbar[i] = Wh[i] * (rho0 + t4 * d * rho0 / 4.0 - t9 * d * rho0 / 16.0);
    }
}

}  // namespace lbf

static int fail(lb_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg; else g_create_error = msg;
    return code;
}

static int cuda_fail(lb_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, LB_ECUDA, m);
}

#define CK(ctx, call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

// Reads the device error word (after the stream has drained); a bounded wait that gave
// up in a kernel is reported as LB_ETIMEOUT and cleared.
static int check_device_error(lb_ctx* c) {
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "D2H");
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (h != 0) {
        CK(c, cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream), "memset");
        return fail(c, LB_ETIMEOUT, "a step kernel gave up waiting for its TMA loads");
    }
    return LB_OK;
}

extern "C" {

size_t lb_workspace_bytes(int nx, int ny, int precision) {
    Grid g;
    const int es = elem_size(precision);
    if (!make_grid(nx, ny, es, &g)) return 0;
    return make_layout(g, es).total;
}

int lb_create(int nx, int ny, int precision, uint64_t seed, double rho0, double cs2, void* workspace,
              size_t workspace_bytes, lb_ctx** out) {
    if (!out) return fail(nullptr, LB_EINVAL, "out is NULL");
    *out = nullptr;
    const int es = elem_size(precision);
    if (es == 0) return fail(nullptr, LB_EINVAL, "precision must be LB_FP32, LB_FP16DEV or LB_FP64");
    Grid g;
    if (!make_grid(nx, ny, es, &g)) return fail(nullptr, LB_EINVAL, "nx and ny must lie in [2, 65536]");
    if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail(nullptr, LB_EINVAL, "rho0 must be positive");
    if (!(cs2 > 0.0) || !std::isfinite(cs2)) return fail(nullptr, LB_EINVAL, "cs2 must be positive");
    lb_ctx* c = new lb_ctx();
    c->nx = nx; c->ny = ny; c->n = (long long)nx * ny; c->precision = precision;
    c->fp16 = precision == LB_FP16DEV ? 1 : 0;
    c->seed = seed; c->rho0 = rho0; c->cs2 = cs2; c->g = g; c->L = make_layout(g, es);
    c->cs2_linear = cs2;
    c->p0_rest = cs2 * rho0;
    c->eos_poly[0] = cs2 * rho0; c->eos_poly[1] = cs2;
    c->eos_cq[0] = cs2;
    c->pow2 = is_pow2(nx) && is_pow2(ny);
    cudaGetDevice(&c->device);
    if (workspace) {
        if (workspace_bytes < c->L.total || ((uintptr_t)workspace & 255)) {
            delete c;
            return fail(nullptr, LB_ENOMEM, "workspace smaller than lb_workspace_bytes() or not 256-byte aligned");
        }
        c->ws = (char*)workspace;
    } else {
        cudaError_t e = cudaMalloc((void**)&c->ws, c->L.total);
        if (e != cudaSuccess) {
            delete c;
            return fail(nullptr, LB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        c->owns = true;
    }
    c->pop[0] = c->ws + c->L.pop[0];
    c->pop[1] = c->ws + c->L.pop[1];
    c->z1 = (float2*)(c->ws + c->L.z1);
    c->z2 = (float2*)(c->ws + c->L.z2);
    c->twx = (float2*)(c->ws + c->L.twx);
    c->twy = (float2*)(c->ws + c->L.twy);
    c->cosx = (float*)(c->ws + c->L.cosx);
    c->cosy = (float*)(c->ws + c->L.cosy);
    c->bins = (double*)(c->ws + c->L.bins);
    c->counts = (unsigned long long*)(c->ws + c->L.counts);
    c->bin16 = (unsigned short*)(c->ws + c->L.bin16);
    c->partial = (double*)(c->ws + c->L.partial);
    c->sums3 = (double*)(c->ws + c->L.sums3);
    c->fbar_dev = (double*)(c->ws + c->L.fbar);
    c->err_dev = (int*)(c->ws + c->L.err);
    rest_populations(rho0, cs2, c->fbar);
    {
        // LBFLUCT_STEP_KERNEL=simple selects the plain kernel; LBFLUCT_TMA_TILE=<0..4> fixes a
        // tile shape (otherwise each step uses the fastest one for its noise mode)
        const char* v = std::getenv("LBFLUCT_STEP_KERNEL");
        c->use_sweep = v && (std::strcmp(v, "sweep") == 0 || std::strcmp(v, "sweep6") == 0) && sweep_fits(g);
        c->sweep_occ6 = v && std::strcmp(v, "sweep6") == 0;
        if (precision == LB_FP64) c->use_sweep = false;
        // FP64 storage runs the plain kernel (its arithmetic is FP64 throughout)
        const bool want_tma = !(v && std::strcmp(v, "simple") == 0) && !c->use_sweep && precision != LB_FP64;
        const char* tv = std::getenv("LBFLUCT_TMA_TILE");
        c->tma_tile_fixed = tv ? std::atoi(tv) : -1;
        if (c->tma_tile_fixed >= tma_tile_count()) c->tma_tile_fixed = -1;
        c->tma_tile = c->tma_tile_fixed >= 0 ? c->tma_tile_fixed : tma_default_tile(LB_NOISE_LW, c->fp16);
        c->use_tma = want_tma && tensor_map_bytes() <= sizeof(c->tmap[0]) &&
                     make_pop_tensor_map(c->pop[0], g, c->tma_tile, c->fp16, c->tmap[0]) &&
                     make_pop_tensor_map(c->pop[1], g, c->tma_tile, c->fp16, c->tmap[1]);
    }

    // host tables in FP64 -> device
    std::vector<float2> tw(std::max(nx, ny));
    std::vector<float> cs(std::max(nx, ny));
    auto upload = [&](int n, float2* dtw, float* dcos) -> cudaError_t {
        for (int k = 0; k < n; ++k) {
            const double a = 2.0 * M_PI * (double)k / n;
            tw[k] = make_float2((float)std::cos(a), (float)-std::sin(a));   // exp(-2 pi i k/n)
        }
        for (int k = 0; k < n; ++k) cs[k] = (float)std::cos(2.0 * M_PI * (double)k / n);
        cudaError_t e = cudaMemcpy(dtw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(dcos, cs.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    };
    cudaError_t e = upload(nx, c->twx, c->cosx);
    if (e == cudaSuccess) e = upload(ny, c->twy, c->cosy);
    if (e == cudaSuccess && precision == LB_FP64) {
        c->twxd = (double2*)(c->ws + c->L.twxd);
        c->twyd = (double2*)(c->ws + c->L.twyd);
        c->cosxd = (double*)(c->ws + c->L.cosxd);
        c->cosyd = (double*)(c->ws + c->L.cosyd);
        std::vector<double2> twd(std::max(nx, ny));
        std::vector<double> csd(std::max(nx, ny));
        for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
            const int n = which == 0 ? nx : ny;
            for (int k = 0; k < n; ++k) {
                const double a = 2.0 * M_PI * (double)k / n;
                twd[k] = make_double2(std::cos(a), -std::sin(a));
                csd[k] = std::cos(a);
            }
            e = cudaMemcpy(which == 0 ? c->twxd : c->twyd, twd.data(), sizeof(double2) * n, cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(which == 0 ? c->cosxd : c->cosyd, csd.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(c->fbar_dev, c->fbar, sizeof(double) * Q, cudaMemcpyHostToDevice);
    // rest state: every deviation (and ghost) zero
    if (e == cudaSuccess) e = cudaMemset(c->pop[0], 0, (size_t)Q * g.plane * es);
    if (e == cudaSuccess) e = cudaMemset(c->pop[1], 0, (size_t)Q * g.plane * es);
    if (e == cudaSuccess) e = cudaMemset(c->bins, 0, 3 * MAX_BINS * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->err_dev, 0, sizeof(int));
    if (e != cudaSuccess) {
        if (c->owns) cudaFree(c->ws);
        delete c;
        return fail(nullptr, LB_ECUDA, std::string("lb_create: ") + cudaGetErrorString(e));
    }
    c->sa.g = g;
    c->sa.rho0 = (float)rho0;
    c->sa.cs2m = (float)(cs2 - SIGMA_S2);
    c->sa.rk = make_round_keys(seed);
    c->sad.g = g;
    c->sad.rho0 = rho0;
    c->sad.cs2m = cs2 - SIGMA_S2;
    c->sad.rk = c->sa.rk;
    *out = c;
    return LB_OK;
}

int lb_destroy(lb_ctx* c) {
    if (!c) return LB_EINVAL;
    DeviceGuard dg(c->device);
    for (auto& p : c->ev) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    if (c->owns) cudaFree(c->ws);
    delete c;
    return LB_OK;
}

int lb_set_stream(lb_ctx* c, void* stream) {
    if (!c) return LB_EINVAL;
    c->stream = (cudaStream_t)stream;
    return LB_OK;
}

int lb_set_params(lb_ctx* c, double kT, double kappa, double tau_s, double tau_b, double tau_ghost, int mode) {
    if (!c) return LB_EINVAL;
    std::string why;
    int r = validate(c->nx, c->ny, c->rho0, c->cs2, kT, kappa, tau_s, tau_b, tau_ghost, mode, &why);
    if (r != LB_OK) return fail(c, r, why);
    if (mode == LB_NOISE_FULL && kT > 0.0 && (!c->pow2 || c->ny > 8192))
        return fail(c, LB_EINVAL, "correlated noise needs nx and ny powers of two and ny <= 8192");
    if (mode == LB_NOISE_FULL && kT > 0.0 && c->precision == LB_FP64 && noise_strip_d(c->nx, c->ny) < 2)
        return fail(c, LB_EINVAL, "correlated noise with FP64 storage needs ny <= 4096");
    c->kT = kT; c->kappa = kappa; c->tau_s = tau_s; c->tau_b = tau_b; c->tau_g = tau_ghost;
    c->noise_mode = mode;
    c->warnings = (kT >= 0.1 * SIGMA_S2 * c->rho0) ? LB_WARN_LOW_MACH : 0;   // Eq. (low-mach)
    StepArgs& a = c->sa;
    a.kappa = (float)kappa;
    a.lb = (float)(-1.0 / tau_b);
    a.ls = (float)(-1.0 / tau_s);
    a.lq = (float)(-1.0 / tau_ghost);
    a.le = (float)(-1.0 / tau_ghost);
    const NoiseCoef nc = noise_coef(c->rho0, c->cs2, kT, kappa, tau_s, tau_b, tau_ghost);
    // Sec. IV: xi = L nu with L L^T = Xi(0) on modes 4..9; only the (4,9) block is coupled
    const double x44 = nc.a44, x49 = (mode == LB_NOISE_DIAG) ? 0.0 : nc.a49, x99 = nc.a99;
    double L44, L49 = 0.0, L94, L99;
    if (c->factor == LB_FACTOR_EIGEN) {
        eigen_factor_2x2(x44, x49, x99, &L44, &L49, &L94, &L99);
    } else {
        L44 = std::sqrt(std::fmax(x44, 0.0));
        L94 = L44 > 0.0 ? x49 / L44 : 0.0;
        L99 = std::sqrt(std::fmax(x99 - L94 * L94, 0.0));
    }
    a.L44 = (float)L44; a.L49 = (float)L49; a.L94 = (float)L94; a.L99 = (float)L99;
    a.s5 = (float)std::sqrt(std::fmax(nc.x55, 0.0));
    a.s6 = (float)std::sqrt(std::fmax(nc.x66, 0.0));
    a.s7 = (float)std::sqrt(std::fmax(nc.x77, 0.0));
    // real-space correlated noise: factors of the (4,9) block at k^2 = 0, 4, 16/3, over 4
    double sL[3][4];
    const double sk[3] = {0.0, S_MID, S_MAX};
    for (int j = 0; j < 3; ++j) {
        const double y44 = nc.a44 + nc.b44 * sk[j], y49 = nc.a49 + nc.b49 * sk[j], y99 = nc.a99 + nc.b99 * sk[j];
        double l11, l12 = 0.0, l21, l22;
        if (c->factor == LB_FACTOR_EIGEN) {
            eigen_factor_2x2(y44, y49, y99, &l11, &l12, &l21, &l22);
        } else {
            l11 = std::sqrt(std::fmax(y44, 0.0));
            l21 = l11 > 0.0 ? y49 / l11 : 0.0;
            l22 = std::sqrt(std::fmax(y99 - l21 * l21, 0.0));
        }
        sL[j][0] = 0.25 * l11; sL[j][1] = 0.25 * l12; sL[j][2] = 0.25 * l21; sL[j][3] = 0.25 * l22;
        for (int q = 0; q < 4; ++q) a.sL[j][q] = (float)sL[j][q];
    }
    NoiseGenArgs& ga = c->ga;
    ga.a44 = (float)nc.a44; ga.b44 = (float)nc.b44;
    ga.a49 = (float)nc.a49; ga.b49 = (float)nc.b49;
    ga.a99 = (float)nc.a99; ga.b99 = (float)nc.b99;
    ga.cosx = c->cosx; ga.cosy = c->cosy; ga.nx = c->nx; ga.ny = c->ny;
    ga.eig = c->factor == LB_FACTOR_EIGEN ? 1 : 0;
    ga.rk = a.rk;
    // the same in FP64 for FP64 storage (no rounding of the parameters to FP32)
    StepArgsD& d = c->sad;
    d.kappa = kappa;
    d.lb = -1.0 / tau_b; d.ls = -1.0 / tau_s; d.lq = -1.0 / tau_ghost; d.le = -1.0 / tau_ghost;
    d.L44 = L44; d.L49 = L49; d.L94 = L94; d.L99 = L99;
    d.s5 = std::sqrt(std::fmax(nc.x55, 0.0));
    d.s6 = std::sqrt(std::fmax(nc.x66, 0.0));
    d.s7 = std::sqrt(std::fmax(nc.x77, 0.0));
    for (int j = 0; j < 3; ++j)
        for (int q = 0; q < 4; ++q) d.sL[j][q] = sL[j][q];
    // noise at the local density and sound speed: Xi(0) entries per unit density as affine
    // functions of c_s^2 (noise_coef at rho0 = 1 and cs2 = 0, 1), and c_s^2 as a function of
    // the density deviation
    {
        const NoiseCoef n0 = noise_coef(1.0, 0.0, kT, kappa, tau_s, tau_b, tau_ghost);
        const NoiseCoef n1 = noise_coef(1.0, 1.0, kT, kappa, tau_s, tau_b, tau_ghost);
        const double lu[9] = {n0.a44, n1.a44 - n0.a44, n0.a49, n1.a49 - n0.a49, n0.a99, n1.a99 - n0.a99,
                              std::sqrt(std::fmax(n0.x55, 0.0)), std::sqrt(std::fmax(n0.x66, 0.0)),
                              std::sqrt(std::fmax(n0.x77, 0.0))};
        for (int q = 0; q < 9; ++q) { a.lu[q] = (float)lu[q]; d.lu[q] = lu[q]; }
        for (int q = 0; q < 4; ++q) { a.cq[q] = (float)c->eos_cq[q]; d.cq[q] = c->eos_cq[q]; }
    }
    NoiseGenArgsD& gd = c->gad;
    gd.a44 = nc.a44; gd.b44 = nc.b44; gd.a49 = nc.a49; gd.b49 = nc.b49; gd.a99 = nc.a99; gd.b99 = nc.b99;
    gd.cosx = c->cosxd; gd.cosy = c->cosyd; gd.nx = c->nx; gd.ny = c->ny;
    gd.eig = ga.eig;
    gd.rk = a.rk;
    c->have_params = true;
    return LB_OK;
}

int lb_set_eos(lb_ctx* c, int eos, double beta, double rhoV, double rhoL) {
    if (!c) return LB_EINVAL;
    if (eos != LB_EOS_LINEAR && eos != LB_EOS_DOUBLE_WELL) return fail(c, LB_EINVAL, "unknown equation of state");
    const double r0 = c->rho0;
    double poly[5] = {0, 0, 0, 0, 0}, cq[4] = {0, 0, 0, 0};
    if (eos == LB_EOS_DOUBLE_WELL) {
        if (!(beta > 0.0) || !std::isfinite(beta) || !(rhoV >= 0.0) || !(rhoL > rhoV) || !std::isfinite(rhoL))
            return fail(c, LB_EINVAL, "the double well needs beta > 0 and 0 <= rhoV < rhoL");
        // f0(rho0 + d) = beta (A + d)^2 (B + d)^2 = beta (c0 + c1 d + d^2)^2, A = rho0 - rhoV,
        // B = rho0 - rhoL; p0 = rho df0/drho - f0 and c_s^2 = rho d2f0/drho2 as polynomials in d
        const double A = r0 - rhoV, B = r0 - rhoL, c0 = A * B, c1 = A + B;
        const double f[5] = {c0 * c0, 2 * c0 * c1, c1 * c1 + 2 * c0, 2 * c1, 1.0};   // f0 / beta
        double df[4], d2f[3];
        for (int j = 0; j < 4; ++j) df[j] = (j + 1) * f[j + 1];
        for (int j = 0; j < 3; ++j) d2f[j] = (j + 1) * df[j + 1];
        for (int j = 0; j < 5; ++j) {
            // (rho0 + d) df - f
            const double v = (j < 4 ? r0 * df[j] : 0.0) + (j >= 1 ? df[j - 1] : 0.0) - f[j];
            poly[j] = beta * v;
        }
        for (int j = 0; j < 4; ++j) cq[j] = beta * ((j < 3 ? r0 * d2f[j] : 0.0) + (j >= 1 ? d2f[j - 1] : 0.0));
    } else {
        poly[0] = c->cs2_linear * r0;
        poly[1] = c->cs2_linear;
        cq[0] = c->cs2_linear;
    }
    DeviceGuard dg(c->device);
    // the state in FP64 with the old rest populations, back with the new ones
    double fb_new[Q];
    rest_populations(r0, poly[0] / r0, fb_new);
    double* stage = (double*)c->z1;
    for (int i = 0; i < Q; ++i) {
        CK(c, launch_get_plane(c->pop[c->cur], c->precision, c->g, i, c->fbar[i], stage, c->stream), "get plane");
        CK(c, launch_set_plane(stage, c->pop[c->cur], c->precision, c->g, i, fb_new[i], c->stream), "set plane");
        c->kernels += 2;
    }
    CK(c, cudaMemcpyAsync(c->fbar_dev, fb_new, sizeof(double) * Q, cudaMemcpyHostToDevice, c->stream), "H2D");
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    for (int i = 0; i < Q; ++i) c->fbar[i] = fb_new[i];
    c->eos = eos;
    c->eos_beta = beta; c->eos_rhoV = rhoV; c->eos_rhoL = rhoL;
    for (int j = 0; j < 5; ++j) c->eos_poly[j] = poly[j];
    for (int j = 0; j < 4; ++j) c->eos_cq[j] = cq[j];
    c->p0_rest = poly[0];
    c->cs2 = poly[1];                        // c_s^2 of the linear theory about rho0
    c->sa.cs2m = (float)(poly[1] - SIGMA_S2);
    c->sad.cs2m = poly[1] - SIGMA_S2;
    c->sa.eos = c->sad.eos = eos == LB_EOS_DOUBLE_WELL ? 1 : 0;
    c->sa.e2 = (float)poly[2]; c->sa.e3 = (float)poly[3]; c->sa.e4 = (float)poly[4];
    c->sad.e2 = poly[2]; c->sad.e3 = poly[3]; c->sad.e4 = poly[4];
    for (int q = 0; q < 4; ++q) { c->sa.cq[q] = (float)cq[q]; c->sad.cq[q] = cq[q]; }
    if (c->have_params) {
        const int r = lb_set_params(c, c->kT, c->kappa, c->tau_s, c->tau_b, c->tau_g, c->noise_mode);
        if (r != LB_OK) {
            c->have_params = false;       // the old noise factors belong to the old equation of state
            return r;
        }
    }
    return LB_OK;
}

int lb_set_noise_factor(lb_ctx* c, int factor) {
    if (!c) return LB_EINVAL;
    if (factor != LB_FACTOR_CHOLESKY && factor != LB_FACTOR_EIGEN) return fail(c, LB_EINVAL, "unknown noise factor");
    c->factor = factor;
    if (c->have_params)
        return lb_set_params(c, c->kT, c->kappa, c->tau_s, c->tau_b, c->tau_g, c->noise_mode);
    return LB_OK;
}

static int record_timing(lb_ctx* c, cudaEvent_t* start, cudaEvent_t* stop) {
    if (c->ev_used == c->ev.size()) {
        if (c->ev.size() >= 1024) {
            // fold the finished pairs into the running total and reuse them
            CK(c, cudaEventSynchronize(c->ev.back().second), "cudaEventSynchronize");
            for (auto& p : c->ev) {
                float ms = 0.f;
                CK(c, cudaEventElapsedTime(&ms, p.first, p.second), "cudaEventElapsedTime");
                c->ms_acc += ms;
            }
            c->ev_used = 0;
        } else {
            cudaEvent_t a, b;
            CK(c, cudaEventCreate(&a), "cudaEventCreate");
            CK(c, cudaEventCreate(&b), "cudaEventCreate");
            c->ev.push_back({a, b});
        }
    }
    *start = c->ev[c->ev_used].first;
    *stop = c->ev[c->ev_used].second;
    c->ev_used++;
    return LB_OK;
}

int lb_step(lb_ctx* c, int64_t nsteps) {
    if (!c) return LB_EINVAL;
    if (nsteps < 0) return fail(c, LB_EINVAL, "nsteps must be >= 0");
    if (!c->have_params) return fail(c, LB_ESTATE, "lb_set_params must be called before lb_step");
    DeviceGuard dg(c->device);
    const bool noisy = c->noise_mode != LB_NOISE_OFF && c->kT > 0.0;
    // kernel noise mode: 0 none, 1 uncorrelated, 2 correlated (k-space field), 3 correlated
    // built in real space, 4 uncorrelated at the local density
    const int kmode = !noisy ? 0
                      : (c->noise_mode == LB_NOISE_FULL ? 2
                         : (c->noise_mode == LB_NOISE_FULL_RS ? 3 : (c->noise_mode == LB_NOISE_LW_LOCAL ? 4 : 1)));
    if (kmode == 2 && !c->pow2)
        return fail(c, LB_EINVAL, "correlated noise needs nx and ny powers of two (radix-2 FFT)");
    for (int64_t k = 0; k < nsteps; ++k) {
        const uint32_t tlo = (uint32_t)((uint64_t)c->t & 0xffffffffu), thi = (uint32_t)((uint64_t)c->t >> 32);
        if (c->precision == LB_FP64) {
            // FP64 storage: FP64 noise synthesis and the plain kernel in FP64
            if (kmode == 2) {
                NoiseGenArgsD gd = c->gad;
                gd.t_lo = tlo; gd.t_hi = thi;
                CK(c, launch_noise49_d(reinterpret_cast<double2*>(c->z1), gd, c->twxd, c->twyd, c->stream),
                   "correlated noise");
                c->kernels += 2;
            }
            StepArgsD d = c->sad;
            d.src = c->pop[c->cur];
            d.dst = c->pop[c->cur ^ 1];
            d.xi49 = reinterpret_cast<const double2*>(c->z1);
            d.t_lo = tlo; d.t_hi = thi;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            const bool tm = c->timing > 0 && (c->timing_seq++ % c->timing) == 0;
            if (tm) {
                int r = record_timing(c, &e0, &e1);
                if (r != LB_OK) return r;
                CK(c, cudaEventRecord(e0, c->stream), "cudaEventRecord");
            }
            CK(c, launch_step_simple_d(d, kmode, c->stream), "step kernel launch");
            c->kernels += 1;
            if (tm) {
                CK(c, cudaEventRecord(e1, c->stream), "cudaEventRecord");
                c->launches_acc++;
            }
            c->cur ^= 1;
            c->t++;
            if (c->every > 0 && c->t % c->every == 0) {
                CK(c, launch_stats_sample(c->pop[c->cur], c->precision, c->g, c->z1, c->z2, c->twx, c->twy, c->bin16,
                                          c->bins, c->nbins, c->stream), "spectra sample");
                c->kernels += 6;
                c->nsamples++;
            }
            continue;
        }
        if (kmode == 2) {
            NoiseGenArgs ga = c->ga;
            ga.t_lo = tlo; ga.t_hi = thi;
            CK(c, launch_noise49(c->z1, c->z2, ga, c->twx, c->twy, c->stream), "correlated noise");
            c->kernels += 2;
        }
        StepArgs a = c->sa;
        a.src = c->pop[c->cur];
        a.dst = c->pop[c->cur ^ 1];
        a.xi49 = c->z1;
        a.t_lo = tlo; a.t_hi = thi;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        const bool tm = c->timing > 0 && (c->timing_seq++ % c->timing) == 0;
        if (tm) {
            int r = record_timing(c, &e0, &e1);
            if (r != LB_OK) return r;
            CK(c, cudaEventRecord(e0, c->stream), "cudaEventRecord");
        }
        // the double-well equation of state runs on the TMA kernel's double-well variant (FP32
        // storage, the default tile of the noise mode) or on the plain kernel; the sweep kernel
        // has the noise modes 0..2 only
        const bool poly = c->eos == LB_EOS_DOUBLE_WELL;
        if (c->use_sweep && kmode < 3 && !poly)
            CK(c, launch_step_sweep(a, kmode, c->fp16, c->sweep_occ6, c->stream), "step kernel launch");
        else if (c->use_tma && (!poly || !c->fp16)) {
            const int want = (c->tma_tile_fixed >= 0 && !poly) ? c->tma_tile_fixed : tma_default_tile(kmode, c->fp16);
            if (want != c->tma_tile) {
                // tensor maps are host-encoded descriptors passed by value: re-encode for the shape
                if (!make_pop_tensor_map(c->pop[0], c->g, want, c->fp16, c->tmap[0]) ||
                    !make_pop_tensor_map(c->pop[1], c->g, want, c->fp16, c->tmap[1]))
                    return fail(c, LB_ECUDA, "tensor map encoding failed");
                c->tma_tile = want;
            }
            CK(c, launch_step_tma(a, c->tmap[c->cur], c->err_dev, kmode, c->tma_tile, c->fp16, c->stream, poly),
               "step kernel launch");
        } else
            CK(c, launch_step_simple(a, kmode, c->fp16, c->stream), "step kernel launch");
        c->kernels += 1;
        if (tm) {
            CK(c, cudaEventRecord(e1, c->stream), "cudaEventRecord");
            c->launches_acc++;
        }
        c->cur ^= 1;
        c->t++;
        if (c->every > 0 && c->t % c->every == 0) {
            CK(c, launch_stats_sample(c->pop[c->cur], c->precision, c->g, c->z1, c->z2, c->twx, c->twy, c->bin16,
                                      c->bins, c->nbins, c->stream), "spectra sample");
            c->kernels += 6;
            c->nsamples++;
        }
    }
    return LB_OK;
}

int lb_get_time(lb_ctx* c, int64_t* t) {
    if (!c || !t) return LB_EINVAL;
    *t = c->t;
    return LB_OK;
}

int lb_set_populations(lb_ctx* c, const double* f, int loc, int64_t t) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE) || t < 0) return LB_EINVAL;
    DeviceGuard dg(c->device);
    double* stage = (double*)c->z1;     // n doubles of scratch
    for (int i = 0; i < Q; ++i) {
        const double* src = f + (long long)i * c->n;
        if (loc == LB_HOST) {
            CK(c, cudaMemcpyAsync(stage, src, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream), "H2D");
            src = stage;
        }
        CK(c, launch_set_plane(src, c->pop[c->cur], c->precision, c->g, i, c->fbar[i], c->stream), "set populations");
        c->kernels += 1;
    }
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    c->t = t;
    return LB_OK;
}

int lb_get_populations(lb_ctx* c, double* f, int loc) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE)) return LB_EINVAL;
    DeviceGuard dg(c->device);
    double* stage = (double*)c->z1;
    for (int i = 0; i < Q; ++i) {
        double* dst = (loc == LB_HOST) ? stage : f + (long long)i * c->n;
        CK(c, launch_get_plane(c->pop[c->cur], c->precision, c->g, i, c->fbar[i], dst, c->stream), "get populations");
        c->kernels += 1;
        if (loc == LB_HOST)
            CK(c, cudaMemcpyAsync(f + (long long)i * c->n, stage, sizeof(double) * c->n, cudaMemcpyDeviceToHost,
                                  c->stream), "D2H");
    }
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return check_device_error(c);
}

int lb_moments(lb_ctx* c, double* m, int loc, double sums[3]) {
    if (!c || (m && loc != LB_HOST && loc != LB_DEVICE)) return LB_EINVAL;
    DeviceGuard dg(c->device);
    if (m) {
        double* stage = (double*)c->z1;
        for (int a = 0; a < Q; ++a) {
            double* dst = (loc == LB_HOST) ? stage : m + (long long)a * c->n;
            CK(c, launch_moment(c->pop[c->cur], c->precision, c->g, a, c->fbar_dev, dst, c->stream), "moments");
            c->kernels += 1;
            if (loc == LB_HOST)
                CK(c, cudaMemcpyAsync(m + (long long)a * c->n, stage, sizeof(double) * c->n, cudaMemcpyDeviceToHost,
                                      c->stream), "D2H");
        }
    }
    if (sums) {
        CK(c, launch_sums(c->pop[c->cur], c->precision, c->g, c->fbar_dev, c->partial, c->sums3, c->stream), "sums");
        c->kernels += 2;
        CK(c, cudaMemcpyAsync(sums, c->sums3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
    }
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return check_device_error(c);
}

int lb_set_sampling(lb_ctx* c, int every, int nbins) {
    if (!c) return LB_EINVAL;
    if (every < 0) return fail(c, LB_EINVAL, "every must be >= 0");
    DeviceGuard dg(c->device);
    if (every == 0) {
        c->every = 0;
        return LB_OK;
    }
    if (!c->pow2) return fail(c, LB_EINVAL, "spectra need nx and ny powers of two (radix-2 FFT)");
    if (nbins < 1 || nbins > MAX_BINS) return fail(c, LB_EINVAL, "nbins must lie in [1, 4096]");
    c->every = every;
    c->nbins = nbins;
    c->nsamples = 0;
    CK(c, cudaMemsetAsync(c->bins, 0, 3 * MAX_BINS * sizeof(double), c->stream), "memset");
    CK(c, launch_bin_counts(c->nx, c->ny, nbins, c->bin16, c->counts, c->stream), "bin counts");
    c->kernels += 1;
    c->hcounts.assign(nbins, 0);
    CK(c, cudaMemcpyAsync(c->hcounts.data(), c->counts, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost,
                          c->stream), "D2H");
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_structure_factor(lb_ctx* c, int nbins, double* S_rho, double* S_jl, double* S_jt, int64_t* counts,
                        int64_t* nsamples) {
    if (!c) return LB_EINVAL;
    if (c->every == 0 && c->nbins == 0) return fail(c, LB_ESTATE, "sampling was never turned on");
    if (nbins != c->nbins) return fail(c, LB_EINVAL, "nbins differs from lb_set_sampling");
    DeviceGuard dg(c->device);
    std::vector<double> h(3 * (size_t)nbins);
    CK(c, cudaMemcpyAsync(h.data(), c->bins, sizeof(double) * nbins, cudaMemcpyDeviceToHost, c->stream), "D2H");
    CK(c, cudaMemcpyAsync(h.data() + nbins, c->bins + nbins, sizeof(double) * nbins, cudaMemcpyDeviceToHost,
                          c->stream), "D2H");
    CK(c, cudaMemcpyAsync(h.data() + 2 * nbins, c->bins + 2 * nbins, sizeof(double) * nbins, cudaMemcpyDeviceToHost,
                          c->stream), "D2H");
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    for (int b = 0; b < nbins; ++b) {
        const double den = (double)c->hcounts[b] * (double)c->nsamples;
        if (S_rho) S_rho[b] = den > 0 ? h[b] / den : 0.0;
        if (S_jl) S_jl[b] = den > 0 ? h[nbins + b] / den : 0.0;
        if (S_jt) S_jt[b] = den > 0 ? h[2 * nbins + b] / den : 0.0;
        if (counts) counts[b] = (int64_t)c->hcounts[b];
    }
    if (nsamples) *nsamples = c->nsamples;
    return LB_OK;
}

int lb_warnings(lb_ctx* c) { return c ? c->warnings : 0; }

const char* lb_last_error(lb_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int lb_synchronize(lb_ctx* c) {
    if (!c) return LB_EINVAL;
    DeviceGuard dg(c->device);
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return check_device_error(c);
}

int lb_set_kernel_timing(lb_ctx* c, int on) {
    if (!c) return LB_EINVAL;
    if (on < 0) return fail(c, LB_EINVAL, "timing stride must be >= 0");
    c->timing = on;
    c->timing_seq = 0;
    c->ev_used = 0;
    c->ms_acc = 0.0;
    c->launches_acc = 0;
    return LB_OK;
}

int lb_kernel_time(lb_ctx* c, double* ms, int64_t* launches) {
    if (!c) return LB_EINVAL;
    DeviceGuard dg(c->device);
    double total = c->ms_acc;
    if (c->ev_used > 0) {
        CK(c, cudaEventSynchronize(c->ev[c->ev_used - 1].second), "cudaEventSynchronize");
        for (size_t k = 0; k < c->ev_used; ++k) {
            float v = 0.f;
            CK(c, cudaEventElapsedTime(&v, c->ev[k].first, c->ev[k].second), "cudaEventElapsedTime");
            total += v;
        }
    }
    if (ms) *ms = total;
    if (launches) *launches = c->launches_acc;
    return LB_OK;
}

int lb_launch_count(lb_ctx* c, int64_t* launches) {
    if (!c || !launches) return LB_EINVAL;
    *launches = c->kernels;
    return LB_OK;
}

int lb_noise_matrix(double rho0, double cs2, double kT, double kappa, double tau_s, double tau_b,
                    double tau_ghost, double kx, double ky, double* xi) {
    if (!xi) return LB_EINVAL;
    const NoiseCoef c = noise_coef(rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost);
    const double s = k2_lattice(kx, ky);
    for (int k = 0; k < 81; ++k) xi[k] = 0.0;
    xi[3 * 9 + 3] = c.a44 + c.b44 * s;
    xi[3 * 9 + 8] = xi[8 * 9 + 3] = c.a49 + c.b49 * s;
    xi[8 * 9 + 8] = c.a99 + c.b99 * s;
    xi[4 * 9 + 4] = c.x55;
    xi[5 * 9 + 5] = c.x66;
    xi[6 * 9 + 6] = xi[7 * 9 + 7] = c.x77;
    return LB_OK;
}

int lb_check_params(int nx, int ny, double rho0, double cs2, double kT, double kappa, double tau_s,
                    double tau_b, double tau_ghost, int noise_mode) {
    Grid g;
    if (!make_grid(nx, ny, 4, &g)) return LB_EINVAL;
    return validate(nx, ny, rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode, nullptr);
}

}  // extern "C"
