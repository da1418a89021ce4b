// lb_internal.cuh -- definitions shared by the library's translation units.
//
// Population storage: FP32 deviations df_i = f_i - fbar_i of the POST-collision
// populations f*_i(r, t-1), one plane per velocity i.  The pre-collision state of
// [GACV] Eq. (fluct-lin-lbe) is recovered by pulling: f_i(r, t) = f*_i(r - c_i, t-1).
// Each plane carries GX ghost columns and GY ghost rows on every side that hold
// periodic copies, so every read of the step (r - c_i for nodes up to one cell
// outside the lattice) is an in-bounds, wrap-free address.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>

namespace lbf {

constexpr int Q = 9;
constexpr int GY = 2;    // ghost rows per side
constexpr int MAX_BINS = 4096;

struct Grid {
    int nx, ny;
    int gx;              // ghost columns per side: 128 bytes of elements, so column 0 is 128-byte aligned
    int pitch;           // elements per stored row (>= nx + 2 gx, a multiple of 128 bytes)
    long long plane;     // elements per population plane
    __host__ __device__ __forceinline__ long long at(int x, int y) const {
        return (long long)(y + GY) * pitch + (x + gx);
    }
};

// Storage of one population deviation df_i = f_i - fbar_i.  FP32 keeps df_i; FP16 keeps
// df_i / w_i, which is of the size of the density fluctuation for every i and so stays in
// FP16's normal range.  Arithmetic is FP32 either way.
template <typename T>
struct Elem;

template <>
struct Elem<float> {
    static constexpr int XO = 4;     // elements per 16 bytes (TMA x alignment)
    static constexpr int GW = 8;     // elements per 32-byte sector (ghost column width)
    __host__ __device__ static __forceinline__ float load(float v, int) { return v; }
    __host__ __device__ static __forceinline__ float store(float v, int) { return v; }
};

template <>
struct Elem<__half> {
    static constexpr int XO = 8;
    static constexpr int GW = 16;
    __device__ static __forceinline__ float load(__half v, int i) {
        return __half2float(v) * (i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f));
    }
    __device__ static __forceinline__ __half store(float v, int i) {
        return __float2half_rn(v * (i == 0 ? 2.25f : (i < 5 ? 9.0f : 36.0f)));
    }
    // the stored value itself, g_i = df_i / w_i (kernels that collide in that form)
    __device__ static __forceinline__ float load_g(__half v) { return __half2float(v); }
    __device__ static __forceinline__ __half store_g(float g) { return __float2half_rn(g); }
};

// FP64 storage: deviations in FP64, arithmetic in FP64.
template <>
struct Elem<double> {
    static constexpr int XO = 2;
    static constexpr int GW = 4;
    __host__ __device__ static __forceinline__ double load(double v, int) { return v; }
    __host__ __device__ static __forceinline__ double store(double v, int) { return v; }
};

// arithmetic type of a storage type, and its complex pair
template <typename T>
struct Arith {
    using type = float;
    using vec2 = float2;
};
template <>
struct Arith<double> {
    using type = double;
    using vec2 = double2;
};

// Philox4x32-10 round keys: round r uses (k0 + r W0, k1 + r W1) mod 2^32, computed once on
// the host so that every round is two wide multiplies and two three-input XORs.
struct RoundKeys {
    uint32_t k[20];
};

inline RoundKeys make_round_keys(uint64_t seed) {
    RoundKeys rk;
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0;
        rk.k[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return rk;
}

// Arguments of the fused step kernel (by value), in the arithmetic type R.
template <typename R>
struct StepArgsT {
    Grid g;
    const void* __restrict__ src;    // post-collision deviations at t-1 (planes 0..8, storage type)
    void* __restrict__ dst;          // post-collision deviations at t
    const typename Arith<R>::vec2* __restrict__ xi49;   // FULL mode: (xi_4, xi_9)(r) for this step, [y][x]
    R rho0;
    R cs2m;                          // cs2 - sigma_s^2
    R kappa;
    R lb, ls, lq, le;                // lambda_b, lambda_s, lambda_q, lambda_eps
    R L44, L49, L94, L99;            // factor of the (4,9) block of Xi(0) (L49 = 0: Cholesky)
    R s5, s6, s7;                    // sqrt(Xi_55), sqrt(Xi_66), sqrt(Xi_77) = sqrt(Xi_88)
    R sL[3][4];                      // real-space correlated noise: factors (L44, L49, L94, L99) / 4
                                     // of the (4,9) block of Xi at lattice k^2 = 0, 4, 16/3
    int eos;                         // 0: p0 = cs2 rho; 1: polynomial (double-well) bulk pressure,
                                     // stepped by the plain kernel (lb_step.cu)
    R e2, e3, e4;                    // p0(rho0 + d) - p0(rho0) = d (cs2m + sigma_s^2) + d^2 (e2 + d (e3 + d e4))
    R cq[4];                         // local c_s^2(rho0 + d) = cq0 + d (cq1 + d (cq2 + d cq3))
    R lu[9];                         // local Xi(0): x44 = rho (lu0 + lu1 c), x49 = rho (lu2 + lu3 c),
                                     // x99 = rho (lu4 + lu5 c); lu6..8 = sqrt(x55, x66, x77 / rho)
    uint32_t t_lo, t_hi;
    RoundKeys rk;
};
using StepArgs = StepArgsT<float>;
using StepArgsD = StepArgsT<double>;

// k-space synthesis of the correlated (4,9) noise: Xi_ab(k) = a_ab + b_ab s(k) with s
// the lattice k^2 of [GACV] Appendix B, coefficients computed on the host in FP64.  Key is
// the Philox key form (RoundKeys precomputed, or KeyPair expanded on the fly).
template <typename Key, typename R = float>
struct NoiseGenT {
    R a44, b44, a49, b49, a99, b99;
    int eig;             // 0: Cholesky factor of the (4,9) block, 1: eigen-decomposition factor
    const R* cosx;       // cos(2 pi m / nx), m < nx
    const R* cosy;       // cos(2 pi m / ny), m < ny
    int nx, ny;
    uint32_t t_lo, t_hi;
    Key rk;
};

// ---------------------------------------------------------------------------
// Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk.k[2 * r + 1], (uint32_t)p0);
    }
    return c;
}

// The same generator keyed by a (k0, k1) pair, the round keys formed on the fly.
struct KeyPair {
    uint32_t k0, k1;
};

// Round keys as five 16-byte words, q[j] = keys of rounds 2j and 2j + 1: a record in shared
// memory serves them with five vector loads.
struct __align__(16) RoundKeys4 {
    uint4 q[5];
};

__device__ __forceinline__ RoundKeys4 round_keys4(uint32_t k0, uint32_t k1) {
    RoundKeys4 rk;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        rk.q[j] = make_uint4(k0, k1, k0 + 0x9E3779B9u, k1 + 0xBB67AE85u);
        k0 += 2u * 0x9E3779B9u;
        k1 += 2u * 0xBB67AE85u;
    }
    return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys4& rk) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const uint4 kk = rk.q[j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t ka = h ? kk.z : kk.x, kb = h ? kk.w : kk.y;
            const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
            const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
            c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ ka, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ kb, (uint32_t)p0);
        }
    }
    return c;
}

using NoiseGenArgs = NoiseGenT<RoundKeys>;   // single lattice: round keys precomputed
using NoiseGenArgsD = NoiseGenT<RoundKeys, double>;   // FP64 storage

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const KeyPair& kp) {
    uint32_t k0 = kp.k0, k1 = kp.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Box-Muller is evaluated with the hardware approximations of log2, sqrt, sin and cos
// (absolute error below 1e-6 in the normal except for u1 within ~1e-6 of 1, where r itself
// is below 1.5e-3 and the error below 7e-4).  The uniforms are built exactly from bits:
// x = 1 + (k + 1/2) 2^-20 with k in the top mantissa bits, then u1 = x - 1, exact by
// Sterbenz's lemma; likewise u2 - 1/2 = (1 + (j + 1/2) 2^-12) - 3/2.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One Philox output word -> one Box-Muller pair: the top 20 bits give the radius uniform
// u1 = (k + 1/2) 2^-20, the low 12 bits the angle uniform u2 = (j + 1/2) 2^-12, both built
// exactly from the bits; (n0, n1) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2), evaluated
// as -r (cos, sin)(2 pi (u2 - 1/2)) so that the hardware sine and cosine see |x| < pi.
__device__ __forceinline__ float2 gauss_pair(uint32_t w) {
    const float u1 = __uint_as_float(((w >> 12) << 3) | 0x3f800004u) - 1.0f;
    const float v2 = __uint_as_float(((w & 0xfffu) << 11) | 0x3f800400u) - 1.5f;
    const float l = fmaxf(-1.3862943611198906f * __log2f(u1), 0.0f);     // -2 ln u1 = -2 ln2 log2 u1
    const float r = sqrt_approx(l);
    const float th = 6.2831853071795865f * v2;
    return make_float2(-r * __cosf(th), -r * __sinf(th));
}

// The same pair in FP64 (storage LB_FP64): IEEE log, sqrt and sincos, the form of the
// definition itself.
__device__ __forceinline__ double2 gauss_pair_d(uint32_t w) {
    const double u1 = ((double)(w >> 12) + 0.5) * (1.0 / 1048576.0);
    const double u2 = ((double)(w & 0xfffu) + 0.5) * (1.0 / 4096.0);
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincos(6.283185307179586476925286766559 * u2, &sn, &cs);
    return make_double2(r * cs, r * sn);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// reciprocal in the arithmetic type: hardware approximation in FP32, IEEE in FP64
__device__ __forceinline__ float recip(float x) { return rcp_approx(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// normals of one Philox word in the arithmetic type (same bit layout in both, lb_internal.cuh)
__device__ __forceinline__ void gauss_word(uint32_t w, float* n0, float* n1) {
    const float2 g = gauss_pair(w);
    *n0 = g.x;
    *n1 = g.y;
}
__device__ __forceinline__ void gauss_word(uint32_t w, double* n0, double* n1) {
    const double2 g = gauss_pair_d(w);
    *n0 = g.x;
    *n1 = g.y;
}

// square root in the arithmetic type: hardware approximation in FP32, IEEE in FP64
__device__ __forceinline__ float sqrt_fast(float x) { return sqrt_approx(x); }
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }

// noise draw tags (fourth counter word)
constexpr uint32_t TAG_NODE = 0;     // per node: words 0, 1 -> nu_5..nu_8, word 2 -> (nu_4, nu_9)
constexpr uint32_t TAG_KSPACE = 2;   // per wavevector pair: words 0, 1 -> eta_1(k), eta_2(k)
constexpr uint32_t TAG_STENCIL = 3;  // per node: word w -> white 2-vector field w (++, +-, -+, --)

// Real-space correlated noise (LB_NOISE_FULL_RS).  The (4,9) noise at r is
//   xi(r) = h00(r) + h10(r - e_x) + h01(r - e_y) + h11(r - e_x - e_y),
// where node q contributes h_d(q) = 1/4 sum_ab a^dx b^dy L_ab nu_ab(q): the four white
// 2-vectors nu_ab(q) of its tag-3 draw, times the factors L_ab of Xi at lattice k^2 = 0
// (++), 4 (+- and -+) and 16/3 (--), combined with the 2 x 2 Hadamard signs.  sL holds
// L_ab / 4; h[0..7] = (h00, h10, h01, h11) as (xi_4, xi_9) pairs.
template <typename Args, typename R>
__device__ __forceinline__ void stencil_h(const Args& a, uint32_t node, R h[8]) {
    const uint4 w = philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_STENCIL), a.rk);
    R g[4][2];
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        R n0, n1;
        gauss_word(ww[f], &n0, &n1);
        const int k = f == 0 ? 0 : (f == 3 ? 2 : 1);
        g[f][0] = a.sL[k][0] * n0 + a.sL[k][1] * n1;
        g[f][1] = a.sL[k][2] * n0 + a.sL[k][3] * n1;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const R u = g[0][c] + g[1][c], v = g[0][c] - g[1][c];
        const R wv = g[2][c] + g[3][c], z = g[2][c] - g[3][c];
        h[0 + c] = u + wv;       // h00: all signs +
        h[2 + c] = u - wv;       // h10: sign a
        h[4 + c] = v + z;        // h01: sign b
        h[6 + c] = v - z;        // h11: sign a b
    }
}

// Writes v at (x, y) of a plane and at the ghost copies that (x, y) feeds.  Only columns
// -2, -1, nx, nx+1 and rows -2, -1, ny, ny+1 are ever read, but the ghost columns are
// written GW wide (one 32-byte sector): the eight (FP32) or sixteen (FP16) lanes of a warp
// at an x edge then fill a whole sector instead of a part of one, which spares the memory
// system a read-modify-write of the sector.
template <typename T>
__device__ __forceinline__ void store_with_ghosts(T* plane, const Grid& g, int x, int y, T v) {
    constexpr int GW = Elem<T>::GW;
    const long long c = g.at(x, y);
    plane[c] = v;
    const int dxl = (x < GW) ? g.nx : 0;            // copy to x + nx
    const int dxr = (x >= g.nx - GW) ? -g.nx : 0;   // copy to x - nx
    const int dyb = (y < 2) ? g.ny : 0;
    const int dyt = (y >= g.ny - 2) ? -g.ny : 0;
    if ((dxl | dxr | dyb | dyt) == 0) return;
    const int dxs[3] = {0, dxl, dxr};
    const int dys[3] = {0, dyb, dyt};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if ((a == 0 && b == 0) || (a > 0 && dxs[a] == 0) || (b > 0 && dys[b] == 0)) continue;
            plane[c + dxs[a] + (long long)dys[b] * g.pitch] = v;
        }
    }
}

// Stores the nine planes of one node (converted to the storage type), and its periodic
// ghost copies near an edge.  A node feeds at most one ghost column, one ghost row and
// their corner unless the lattice is narrower than 2 GW or lower than 4 rows; the common
// case is three predicated stores per plane with offsets formed once per node, the rare
// one goes through store_with_ghosts.
template <typename T, typename R, bool GF = false>
__device__ __forceinline__ void store9(T* dst, long long P, const Grid& g, int x, int y, const R o[Q]) {
    constexpr int GW = Elem<T>::GW;
    auto conv = [](R v, int i) -> T {
        if constexpr (GF) return Elem<T>::store_g(v);
        else return Elem<T>::store(v, i);
    };
    const long long c = g.at(x, y);
    const bool xl = x < GW, xr = x >= g.nx - GW, yb = y < 2, yt = y >= g.ny - 2;
    if (!(xl | xr | yb | yt)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) dst[i * P + c] = conv(o[i], i);
    } else if ((xl & xr) | (yb & yt)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) store_with_ghosts(dst + i * P, g, x, y, conv(o[i], i));
    } else {
        const bool hx = xl | xr, hy = yb | yt;
        const long long dx = xl ? (long long)g.nx : (xr ? -(long long)g.nx : 0);
        const long long dy = (yb ? (long long)g.ny : (yt ? -(long long)g.ny : 0)) * g.pitch;
        const long long dxy = dx + dy;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T v = conv(o[i], i);
            T* p = dst + i * P + c;
            p[0] = v;
            if (hx) p[dx] = v;
            if (hy) p[dy] = v;
            if (hx & hy) p[dxy] = v;
        }
    }
}

// Makes `dev` the current device for the lifetime of the guard (the entry points of an
// object created on one device may be called while another device is current).
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() { if (changed) cudaSetDevice(prev); }
};

// Grid of a persistent launch (resident CTAs per SM x SMs) for one kernel, kept per
// device: the first launch on a device raises the kernel's dynamic shared-memory limit
// there and asks the occupancy calculator; later launches read the cached value.  Safe
// to call from several host threads.
constexpr int MAX_DEVICES = 64;
struct GridCache {
    std::atomic<int> grid[MAX_DEVICES];
    std::mutex mu;
};

template <typename K>
cudaError_t resident_grid(K kern, int threads, int smem, GridCache& c, int* grid) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    int g = c.grid[dev].load(std::memory_order_acquire);
    if (g == 0) {
        std::lock_guard<std::mutex> lk(c.mu);
        g = c.grid[dev].load(std::memory_order_relaxed);
        if (g == 0) {
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
                return e;
            int sms = 0, per = 0;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem)) != cudaSuccess)
                return e;
            g = sms * (per > 0 ? per : 1);
            c.grid[dev].store(g, std::memory_order_release);
        }
    }
    *grid = g;
    return cudaSuccess;
}

}  // namespace lbf

// Launchers implemented in the .cu files (host side).
namespace lbf {
cudaError_t launch_step_simple(const StepArgs& a, int noise_mode, int fp16, cudaStream_t s);
cudaError_t launch_step_simple_d(const StepArgsD& a, int noise_mode, cudaStream_t s);
cudaError_t launch_step_sweep(const StepArgs& a, int noise_mode, int fp16, int occ6, cudaStream_t s);
bool sweep_fits(const Grid& g);
cudaError_t launch_step_tma(const StepArgs& a, const void* src_map, int* err, int noise_mode, int tile, int fp16,
                            cudaStream_t s, bool poly = false);
bool make_pop_tensor_map(const void* buf, const Grid& g, int tile, int fp16, void* map_out);
int tma_tile_count();
int tma_default_tile(int noise_mode, int fp16);
size_t tensor_map_bytes();
cudaError_t launch_noise49(float2* buf, float2* scratch, const NoiseGenArgs& ga, const float2* twx,
                           const float2* twy, cudaStream_t s);
cudaError_t launch_noise49_d(double2* buf, const NoiseGenArgsD& ga, const double2* twx, const double2* twy,
                             cudaStream_t s);
int noise_strip_d(int nx, int ny);
// storage: 0 FP32, 1 FP16 deviations, 2 FP64 (the spectra themselves are FP32 transforms)
cudaError_t launch_stats_sample(const void* pops, int storage, const Grid& g, float2* z1, float2* z2,
                                const float2* twx, const float2* twy, const unsigned short* bin16, double* bins,
                                int nbins, cudaStream_t s);
cudaError_t launch_bin_counts(int nx, int ny, int nbins, unsigned short* bin16, unsigned long long* counts,
                              cudaStream_t s);
cudaError_t launch_fft2d(float2* data, int nx, int ny, int sign, const float2* twx, const float2* twy,
                         float scale, cudaStream_t s);
cudaError_t launch_set_plane(const double* src, void* pops, int storage, const Grid& g, int i, double fbar,
                             cudaStream_t s);
cudaError_t launch_get_plane(const void* pops, int storage, const Grid& g, int i, double fbar, double* out,
                             cudaStream_t s);
cudaError_t launch_moment(const void* pops, int storage, const Grid& g, int a, const double* fbar9, double* out,
                          cudaStream_t s);
cudaError_t launch_sums(const void* pops, int storage, const Grid& g, const double* fbar9, double* partial,
                        double* out3, cudaStream_t s);
int sums_partial_count();
void set_context_free_error(const std::string& msg);
// rest populations fbar_i of a lattice at density rho0 with p0 = cs2 rho (Table II at u = 0)
void rest_populations(double rho0, double cs2, double fbar[Q]);
// coefficients of the k-dependent (4,9) block of Xi(k), Eq. (noise-yeo), as functions of the
// lattice k^2 s: {a44, b44, a49, b49, a99, b99} with Xi_ab = a_ab + b_ab s
void noise_coefficients(double rho0, double cs2, double kT, double kappa, double tau_s, double tau_b,
                        double tau_ghost, double out[6]);
}  // namespace lbf
