// lb3d.cu -- the fused fluctuating D3Q19 step for sm_103a and the C ABI of lbfluct3d.h.
//
// One launch performs one time step on every node (collision of lb3_collide.cuh, then
// streaming in pull form: f_i(r, t) = f*_i(r - c_i, t - 1)).  A CTA owns a TX x TY tile of
// the (x, y) plane and marches over a run of z planes.  Before it collides plane z it has
// the density deviations of planes z-1, z, z+1 on its tile plus a one-node ring in shared
// memory (three rotating slots); each new plane's densities are summed from the pulled
// populations, so the step reads every population once from DRAM (the re-reads of the
// tile hit L1/L2) and writes it once: 2 x 19 x sizeof(storage) bytes per node.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "lb3_collide.cuh"
#include "lb_internal.cuh"
#include "lbfluct3d.h"

namespace lbf3 {

constexpr double SIGMA_S2 = 1.0 / 3.0;
constexpr uint32_t TAG_A = 4, TAG_B = 5;   // Philox tags of the two draws per node

template <typename R>
struct Step3Args {
    const R* __restrict__ src;    // post-collision deviations at t-1, 19 planes of P nodes
    R* __restrict__ dst;
    int nx, ny, nz, zc;           // zc: planes per CTA
    long long P;                  // nodes per population plane
    Coef3<R> co;
    R sc[Q3];                     // sqrt(Xi_aa) of the modes with a diagonal factor
    R L44, L164, L1616;           // Cholesky factor of the (4,16) block
    uint32_t t_lo, t_hi;
    lbf::RoundKeys rk;
};

// the 19 pulled deviations of node (x, y, z): f_i = src_i(r - c_i), wrapped coordinates
// xm = x-1, xp = x+1 (mod nx) and the row / plane offsets of y-1, y, y+1 and z-1, z, z+1
template <typename R>
__device__ __forceinline__ void pull19(const R* __restrict__ s, long long P, int x, int xm, int xp, long long ym,
                                       long long y0, long long yp, long long zm, long long z0, long long zp,
                                       R f[Q3]) {
    f[0] = s[z0 + y0 + x];
    f[1] = s[P + z0 + y0 + xm];
    f[2] = s[2 * P + z0 + y0 + xp];
    f[3] = s[3 * P + z0 + ym + x];
    f[4] = s[4 * P + z0 + yp + x];
    f[5] = s[5 * P + zm + y0 + x];
    f[6] = s[6 * P + zp + y0 + x];
    f[7] = s[7 * P + z0 + ym + xm];
    f[8] = s[8 * P + z0 + yp + xm];
    f[9] = s[9 * P + z0 + ym + xp];
    f[10] = s[10 * P + z0 + yp + xp];
    f[11] = s[11 * P + zm + ym + x];
    f[12] = s[12 * P + zp + ym + x];
    f[13] = s[13 * P + zm + yp + x];
    f[14] = s[14 * P + zp + yp + x];
    f[15] = s[15 * P + zm + y0 + xm];
    f[16] = s[16 * P + zm + y0 + xp];
    f[17] = s[17 * P + zp + y0 + xm];
    f[18] = s[18 * P + zp + y0 + xp];
}

__device__ __forceinline__ int wrap_lo(int v, int n) { return v < 0 ? v + n : v; }
__device__ __forceinline__ int wrap_hi(int v, int n) { return v >= n ? v - n : v; }

template <typename R>
__device__ __forceinline__ void normals19(const Step3Args<R>& a, uint32_t node, R xi[Q3]) {
    const uint4 ra = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_A), a.rk);
    const uint4 rb = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_B), a.rk);
    R n4, n16, spare;
    lbf::gauss_word(ra.x, &n4, &xi[5]);
    lbf::gauss_word(ra.y, &xi[6], &xi[7]);
    lbf::gauss_word(ra.z, &xi[8], &xi[9]);
    lbf::gauss_word(ra.w, &xi[10], &xi[11]);
    lbf::gauss_word(rb.x, &xi[12], &xi[13]);
    lbf::gauss_word(rb.y, &xi[14], &xi[15]);
    lbf::gauss_word(rb.z, &n16, &xi[17]);
    lbf::gauss_word(rb.w, &xi[18], &spare);
    (void)spare;
#pragma unroll
    for (int q = 5; q < Q3; ++q) xi[q] *= a.sc[q];
    xi[4] = a.L44 * n4;
    xi[16] = a.L164 * n4 + a.L1616 * n16;
}

template <typename R, int MODE, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) step3_kernel(const Step3Args<R> a) {
    constexpr int RX = TX + 2, RY = TY + 2, NT = TX * TY;
    __shared__ R rs[3][RY][RX];
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long P = a.P, nxy = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, nz);
    const int tid = threadIdx.x;
    const R* __restrict__ src = a.src;

    // density deviations of plane zz (any integer in [-1, nz]) on the tile and its ring
    auto density = [&](int zz, int slot) {
        const int zc = wrap_hi(wrap_lo(zz, nz), nz);
        const long long Z0 = zc * nxy;
        const long long Zm = (zc == 0 ? nz - 1 : zc - 1) * nxy, Zp = (zc == nz - 1 ? 0 : zc + 1) * nxy;
        for (int q = tid; q < RX * RY; q += NT) {
            const int ly = q / RX, lx = q - ly * RX;
            int gx = x0 + lx - 1, gy = y0 + ly - 1;
            R v = R(0);
            if (gx <= nx && gy <= ny) {          // gx, gy >= -1 always
                gx = wrap_hi(wrap_lo(gx, nx), nx);
                gy = wrap_hi(wrap_lo(gy, ny), ny);
                const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
                const long long Y0 = (long long)gy * nx;
                const long long Ym = (long long)(gy == 0 ? ny - 1 : gy - 1) * nx;
                const long long Yp = (long long)(gy == ny - 1 ? 0 : gy + 1) * nx;
                R f[Q3];
                pull19(src, P, gx, xm, xp, Ym, Y0, Yp, Zm, Z0, Zp, f);
                v = drho19(f);
            }
            rs[slot][ly][lx] = v;
        }
    };

    density(z0 - 1, 0);
    density(z0, 1);
    const int lx = tid % TX, ly = tid / TX;
    const int x = x0 + lx, y = y0 + ly;
    const bool own = x < nx && y < ny;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const long long Y0 = (long long)y * nx;
    const long long Ym = (long long)(y == 0 ? ny - 1 : y - 1) * nx;
    const long long Yp = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
    for (int z = z0; z < z1; ++z) {
        const int s0 = (z - z0 + 1) % 3, sm = (s0 + 2) % 3, sp = (s0 + 1) % 3;
        density(z + 1, sp);
        __syncthreads();
        if (own) {
            const long long Z0 = (long long)z * nxy;
            const long long Zm = (long long)(z == 0 ? nz - 1 : z - 1) * nxy;
            const long long Zp = (long long)(z == nz - 1 ? 0 : z + 1) * nxy;
            R f[Q3];
            pull19(src, P, x, xm, xp, Ym, Y0, Yp, Zm, Z0, Zp, f);
            const int cx = lx + 1, cy = ly + 1;
            Rho3<R> r;
            r.c = rs[s0][cy][cx];
            r.xp = rs[s0][cy][cx + 1]; r.xm = rs[s0][cy][cx - 1];
            r.yp = rs[s0][cy + 1][cx]; r.ym = rs[s0][cy - 1][cx];
            r.zp = rs[sp][cy][cx]; r.zm = rs[sm][cy][cx];
            r.ap = rs[s0][cy + 1][cx + 1]; r.am = rs[s0][cy - 1][cx - 1];      // (1,1,0)
            r.bp = rs[s0][cy - 1][cx + 1]; r.bm = rs[s0][cy + 1][cx - 1];      // (1,-1,0)
            r.cp = rs[sp][cy + 1][cx]; r.cm = rs[sm][cy - 1][cx];              // (0,1,1)
            r.dp = rs[sm][cy + 1][cx]; r.dm = rs[sp][cy - 1][cx];              // (0,1,-1)
            r.ep = rs[sp][cy][cx + 1]; r.em = rs[sm][cy][cx - 1];              // (1,0,1)
            r.fp = rs[sp][cy][cx - 1]; r.fm = rs[sm][cy][cx + 1];              // (-1,0,1)
            R xi[Q3];
#pragma unroll
            for (int q = 0; q < Q3; ++q) xi[q] = R(0);
            const long long node = Z0 + Y0 + x;
            if (MODE == 1) normals19(a, (uint32_t)node, xi);
            R o[Q3];
            collide19(a.co, f, r, xi, o);
            R* __restrict__ d = a.dst + node;
#pragma unroll
            for (int i = 0; i < Q3; ++i) d[i * P] = o[i];
        }
        __syncthreads();
    }
}

template <typename R, int MODE>
static cudaError_t launch3(const Step3Args<R>& a, dim3 grid, cudaStream_t s) {
    constexpr int TX = 32, TY = 8;
    step3_kernel<R, MODE, TX, TY><<<grid, TX * TY, 0, s>>>(a);
    return cudaGetLastError();
}

// rest populations: w_i 3 cs2 rho0 on the moving velocities, the remainder at rest
static void rest19(double rho0, double cs2, double fbar[Q3]) {
    double moving = 0.0;
    for (int i = 1; i < Q3; ++i) {
        const double w = i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0;
        fbar[i] = w * 3.0 * cs2 * rho0;
        moving += fbar[i];
    }
    fbar[0] = rho0 - moving;
}

static double norm19(int a) {
    static const double N[Q3] = {1, 1.0 / 3, 1.0 / 3, 1.0 / 3, 2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                 2.0 / 3, 2.0 / 3, 2.0 / 3, 2.0 / 9, 2.0 / 9, 2.0 / 9, 2.0, 4.0 / 3, 4.0 / 9};
    return N[a];
}

// Xi(0) in closed form: in the variables y4 = m4 - d rho, y16 = m16 + d rho (d = 3 cs2 - 1)
// the linearised collision is diagonal and the equal-time covariances of the ansatz
// <df_i df_j> = (S/rho0) fbar_i delta_ij (S = rho0 kT / cs2) are rho0 kT (5 - 9 cs2),
// 9 rho0 kT (1 - cs2), 3 rho0 kT (3 cs2 - 1) for (y4, y4), (y16, y16), (y4, y16) and
// N_a rho0 kT / sigma_s^2 for the other non-conserved modes; stationarity under
// m -> (1 + lambda) m + xi gives the entries below.
static void xi_zero19(double rho0, double cs2, double kT, double lb, double ls, double lg, double X[Q3 * Q3]) {
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

template <typename R>
__global__ void set_plane3_kernel(const double* __restrict__ src, R* __restrict__ dst, long long n, double fbar) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = (R)(src[k] - fbar);
}

template <typename R>
__global__ void get_plane3_kernel(const R* __restrict__ src, double* __restrict__ dst, long long n, double fbar) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = (double)src[k] + fbar;
}

// per-block FP64 partial sums of the density and momentum deviations
template <typename R>
__global__ void sums3_kernel(const R* __restrict__ p, long long n, double* __restrict__ partial) {
    double s[4] = {0, 0, 0, 0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double f[Q3];
#pragma unroll
        for (int i = 0; i < Q3; ++i) f[i] = (double)p[i * n + k];
        double r = 0.0;
#pragma unroll
        for (int i = 0; i < Q3; ++i) r += f[i];
        s[0] += r;
        s[1] += (f[1] - f[2]) + (f[7] - f[10]) + (f[8] - f[9]) + (f[15] - f[18]) - (f[16] - f[17]);
        s[2] += (f[3] - f[4]) + (f[7] - f[10]) - (f[8] - f[9]) + (f[11] - f[14]) + (f[12] - f[13]);
        s[3] += (f[5] - f[6]) + (f[11] - f[14]) - (f[12] - f[13]) + (f[15] - f[18]) + (f[16] - f[17]);
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
    int nx = 0, ny = 0, nz = 0, precision = 0, device = 0, es = 4;
    long long n = 0;
    uint64_t seed = 0;
    double rho0 = 1.0, cs2 = 1.0 / 3.0;
    double fbar[Q3] = {};
    char* ws = nullptr;
    void* pop[2] = {nullptr, nullptr};
    double* stage = nullptr;        // one FP64 plane
    double* partial = nullptr;      // SUM3_BLOCKS x 4
    int cur = 0;
    bool have_params = false;
    int noise_mode = LB_NOISE_OFF;
    double kT = 0, kappa = 0;
    Step3Args<float> af{};
    Step3Args<double> ad{};
    dim3 grid;
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

struct Layout3 {
    size_t pop[2], stage, partial, total;
};

Layout3 layout3(long long n, int es) {
    Layout3 L{};
    size_t off = 0;
    for (int k = 0; k < 2; ++k) {
        L.pop[k] = off;
        off = align256(off + (size_t)Q3 * n * es);
    }
    L.stage = off;
    off = align256(off + (size_t)n * sizeof(double));
    L.partial = off;
    off = align256(off + (size_t)SUM3_BLOCKS * 4 * sizeof(double));
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

// the z run of a CTA: enough CTAs for eight per SM, each at least one plane
void choose_grid(lb3_ctx* c) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const long long bxy = (long long)((c->nx + 31) / 32) * ((c->ny + 7) / 8);
    const long long want = 8LL * sms;
    long long chunks = std::max(1LL, std::min((long long)c->nz, (want + bxy - 1) / bxy));
    const int zc = (int)((c->nz + chunks - 1) / chunks);
    chunks = (c->nz + zc - 1) / zc;
    c->grid = dim3((c->nx + 31) / 32, (c->ny + 7) / 8, (unsigned)chunks);
    c->af.zc = c->ad.zc = zc;
}

template <typename R>
void fill_args(lb3_ctx* c, Step3Args<R>* a, double tau_s, double tau_b, double tau_g, const double X[Q3 * Q3],
               double L44, double L164, double L1616) {
    a->nx = c->nx; a->ny = c->ny; a->nz = c->nz; a->P = c->n;
    a->co.rho0 = (R)c->rho0;
    a->co.d = (R)(3.0 * c->cs2 - 1.0);
    a->co.kappa = (R)c->kappa;
    a->co.lb = (R)(-1.0 / tau_b);
    a->co.ls = (R)(-1.0 / tau_s);
    a->co.lg = (R)(-1.0 / tau_g);
    for (int q = 0; q < Q3; ++q) a->sc[q] = (R)(q >= 5 ? std::sqrt(std::max(X[q * Q3 + q], 0.0)) : 0.0);
    a->L44 = (R)L44; a->L164 = (R)L164; a->L1616 = (R)L1616;
    a->rk = lbf::make_round_keys(c->seed);
}

}  // namespace

extern "C" {

size_t lb3_workspace_bytes(int nx, int ny, int nz, int precision) {
    const int es = es_of(precision);
    if (!es || !sizes_ok(nx, ny, nz)) return 0;
    return layout3((long long)nx * ny * nz, es).total;
}

int lb3_create(int nx, int ny, int nz, int precision, uint64_t seed, double rho0, double cs2, lb3_ctx** out) {
    if (!out) return fail3(nullptr, LB_EINVAL, "out is NULL");
    *out = nullptr;
    const int es = es_of(precision);
    if (!es) return fail3(nullptr, LB_EINVAL, "precision must be LB_FP32 or LB_FP64");
    if (!sizes_ok(nx, ny, nz)) return fail3(nullptr, LB_EINVAL, "sizes must be >= 1 with nx*ny*nz < 2^32");
    if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail3(nullptr, LB_EINVAL, "rho0 must be positive");
    if (!(cs2 > 0.0) || !std::isfinite(cs2)) return fail3(nullptr, LB_EINVAL, "cs2 must be positive");
    lb3_ctx* c = new lb3_ctx();
    c->nx = nx; c->ny = ny; c->nz = nz; c->n = (long long)nx * ny * nz;
    c->precision = precision; c->es = es; c->seed = seed; c->rho0 = rho0; c->cs2 = cs2;
    cudaGetDevice(&c->device);
    const Layout3 L = layout3(c->n, es);
    cudaError_t e = cudaMalloc((void**)&c->ws, L.total);
    if (e != cudaSuccess) {
        delete c;
        return fail3(nullptr, LB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->pop[0] = c->ws + L.pop[0];
    c->pop[1] = c->ws + L.pop[1];
    c->stage = (double*)(c->ws + L.stage);
    c->partial = (double*)(c->ws + L.partial);
    rest19(rho0, cs2, c->fbar);
    e = cudaMemset(c->pop[0], 0, (size_t)Q3 * c->n * es);
    if (e == cudaSuccess) e = cudaMemset(c->pop[1], 0, (size_t)Q3 * c->n * es);
    if (e != cudaSuccess) {
        cudaFree(c->ws);
        delete c;
        return fail3(nullptr, LB_ECUDA, std::string("lb3_create: ") + cudaGetErrorString(e));
    }
    choose_grid(c);
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

int lb3_noise_matrix(double rho0, double cs2, double kT, double tau_s, double tau_b, double tau_ghost, double* xi) {
    if (!xi || !(rho0 > 0) || !(cs2 > 0) || kT < 0 || !(tau_s > 0.5) || !(tau_b > 0.5) || !(tau_ghost > 0.5))
        return LB_EINVAL;
    xi_zero19(rho0, cs2, kT, -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_ghost, xi);
    return LB_OK;
}

int lb3_set_params(lb3_ctx* c, double kT, double kappa, double tau_s, double tau_b, double tau_ghost, int mode) {
    if (!c) return LB_EINVAL;
    if (!(tau_s > 0.5) || !(tau_b > 0.5) || !(tau_ghost > 0.5) || !std::isfinite(tau_s) || !std::isfinite(tau_b) ||
        !std::isfinite(tau_ghost))
        return fail3(c, LB_EINVAL, "relaxation times must exceed 1/2");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return fail3(c, LB_EINVAL, "kT must be >= 0");
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) return fail3(c, LB_EINVAL, "kappa must be >= 0");
    if (mode != LB_NOISE_OFF && mode != LB_NOISE_LW)
        return fail3(c, LB_EINVAL, "the D3Q19 lattice takes LB_NOISE_OFF or LB_NOISE_LW");
    double X[Q3 * Q3];
    xi_zero19(c->rho0, c->cs2, kT, -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_ghost, X);
    double L44 = 0, L164 = 0, L1616 = 0;
    if (mode == LB_NOISE_LW && kT > 0) {
        const double x44 = X[4 * Q3 + 4], x416 = X[4 * Q3 + 16], x1616 = X[16 * Q3 + 16];
        const double scale = std::max(std::fabs(x44), std::fabs(x1616));
        const double tol = 1e-12 * scale;
        if (x44 < -tol || x1616 < -tol || x44 * x1616 - x416 * x416 < -tol * scale)
            return fail3(c, LB_ENOTPSD, "Xi(0) is not positive semidefinite (needs cs2 <= 5/9)");
        L44 = x44 > tol ? std::sqrt(x44) : 0.0;
        L164 = L44 > 0 ? x416 / L44 : 0.0;
        L1616 = std::sqrt(std::max(x1616 - L164 * L164, 0.0));
    }
    c->kT = kT;
    c->kappa = kappa;
    c->noise_mode = mode;
    fill_args(c, &c->af, tau_s, tau_b, tau_ghost, X, L44, L164, L1616);
    fill_args(c, &c->ad, tau_s, tau_b, tau_ghost, X, L44, L164, L1616);
    c->have_params = true;
    return LB_OK;
}

int lb3_step(lb3_ctx* c, int64_t nsteps) {
    if (!c) return LB_EINVAL;
    if (nsteps < 0) return fail3(c, LB_EINVAL, "nsteps must be >= 0");
    if (!c->have_params) return fail3(c, LB_ESTATE, "lb3_set_params must be called before lb3_step");
    lbf::DeviceGuard dg(c->device);
    const int kmode = (c->noise_mode == LB_NOISE_LW && c->kT > 0.0) ? 1 : 0;
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
            e = kmode ? launch3<double, 1>(a, c->grid, c->stream) : launch3<double, 0>(a, c->grid, c->stream);
        } else {
            Step3Args<float> a = c->af;
            a.src = (const float*)c->pop[c->cur];
            a.dst = (float*)c->pop[c->cur ^ 1];
            a.t_lo = tlo; a.t_hi = thi;
            e = kmode ? launch3<float, 1>(a, c->grid, c->stream) : launch3<float, 0>(a, c->grid, c->stream);
        }
        if (e != cudaSuccess) return cuda_fail3(c, e, "D3Q19 step kernel launch");
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

static unsigned plane_blocks(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 4096); }

int lb3_set_populations(lb3_ctx* c, const double* f, int loc, int64_t t) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE) || t < 0) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (int i = 0; i < Q3; ++i) {
        const double* src = f + (long long)i * c->n;
        if (loc == LB_HOST) {
            cudaError_t e = cudaMemcpyAsync(c->stage, src, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "H2D");
            src = c->stage;
        }
        if (c->precision == LB_FP64)
            set_plane3_kernel<double><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                src, (double*)c->pop[c->cur] + (long long)i * c->n, c->n, c->fbar[i]);
        else
            set_plane3_kernel<float><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                src, (float*)c->pop[c->cur] + (long long)i * c->n, c->n, c->fbar[i]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail3(c, e, "set populations");
        c->kernels += 1;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    c->t = t;
    return LB_OK;
}

int lb3_get_populations(lb3_ctx* c, double* f, int loc) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE)) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (int i = 0; i < Q3; ++i) {
        double* dst = loc == LB_HOST ? c->stage : f + (long long)i * c->n;
        if (c->precision == LB_FP64)
            get_plane3_kernel<double><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                (const double*)c->pop[c->cur] + (long long)i * c->n, dst, c->n, c->fbar[i]);
        else
            get_plane3_kernel<float><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                (const float*)c->pop[c->cur] + (long long)i * c->n, dst, c->n, c->fbar[i]);
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
    return LB_OK;
}

int lb3_sums(lb3_ctx* c, double sums[4]) {
    if (!c || !sums) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    if (c->precision == LB_FP64)
        sums3_kernel<double><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const double*)c->pop[c->cur], c->n, c->partial);
    else
        sums3_kernel<float><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const float*)c->pop[c->cur], c->n, c->partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail3(c, e, "sums kernel");
    c->kernels += 1;
    std::vector<double> h((size_t)SUM3_BLOCKS * 4);
    e = cudaMemcpyAsync(h.data(), c->partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "sums D2H");
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
    return LB_OK;
}

const char* lb3_last_error(lb3_ctx* c) { return c ? c->err.c_str() : g3_error.c_str(); }

}  // extern "C"
