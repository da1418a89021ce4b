// lb_internal.cuh -- definitions shared by the library's translation units.
//
// Population storage: FP32 deviations df_i = f_i - fbar_i of the POST-collision
// populations f*_i(r, t-1), one plane per velocity i.  The pre-collision state of
// [GACV] Eq. (fluct-lin-lbe) is recovered by pulling: f_i(r, t) = f*_i(r - c_i, t-1).
// Each plane carries GX ghost columns and GY ghost rows on every side that hold
// periodic copies, so every read of the step (r - c_i for nodes up to one cell
// outside the lattice) is an in-bounds, wrap-free address.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbf {

constexpr int Q = 9;
constexpr int GX = 32;   // ghost columns per side: keeps column 0 at a 128-byte boundary
constexpr int GY = 2;    // ghost rows per side
constexpr int MAX_BINS = 4096;

struct Grid {
    int nx, ny;
    int pitch;           // elements per stored row (>= nx + 2 GX, multiple of 32)
    long long plane;     // elements per population plane
    __host__ __device__ __forceinline__ long long at(int x, int y) const {
        return (long long)(y + GY) * pitch + (x + GX);
    }
};

// Arguments of the fused step kernel (by value).
struct StepArgs {
    Grid g;
    const float* __restrict__ src;   // post-collision deviations at t-1 (planes 0..8)
    float* __restrict__ dst;         // post-collision deviations at t
    const float2* __restrict__ xi49; // FULL mode: (xi_4, xi_9)(r) for this step, [y][x]
    float rho0;
    float cs2m;                      // cs2 - sigma_s^2
    float kappa;
    float lb, ls, lq, le;            // lambda_b, lambda_s, lambda_q, lambda_eps
    float L44, L94, L99;             // Cholesky factor of the (4,9) block of Xi(0)
    float s5, s6, s7;                // sqrt(Xi_55), sqrt(Xi_66), sqrt(Xi_77) = sqrt(Xi_88)
    uint32_t key0, key1, t_lo, t_hi;
};

// k-space synthesis of the correlated (4,9) noise: Xi_ab(k) = a_ab + b_ab s(k) with s
// the lattice k^2 of [GACV] Appendix B, coefficients computed on the host in FP64.
struct NoiseGenArgs {
    float a44, b44, a49, b49, a99, b99;
    const float* cosx;   // cos(2 pi m / nx), m < nx
    const float* cosy;   // cos(2 pi m / ny), m < ny
    int nx, ny;
    uint32_t key0, key1, t_lo, t_hi;
};

// ---------------------------------------------------------------------------
// Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Two unit normals by Box-Muller from two 32-bit words.  u = (2k+1) 2^-24 with k the
// top 23 bits is exact in FP32; the angle uses sincospif on 2u (also exact).
__device__ __forceinline__ float2 gauss_pair(uint32_t a, uint32_t b) {
    const float u1 = __uint2float_rn(a >> 9) * 0x1p-23f + 0x1p-24f;
    const float u2 = __uint2float_rn(b >> 9) * 0x1p-23f + 0x1p-24f;
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

// noise draw tags (fourth counter word)
constexpr uint32_t TAG_MODES_5_8 = 0;   // nu_5..nu_8
constexpr uint32_t TAG_MODES_4_9 = 1;   // (nu_4, nu_9)
constexpr uint32_t TAG_KSPACE = 2;      // eta_1(k), eta_2(k)

// Writes v at (x, y) of a plane and at the ghost copies that (x, y) feeds.
__device__ __forceinline__ void store_with_ghosts(float* plane, const Grid& g, int x, int y, float v) {
    const long long c = g.at(x, y);
    plane[c] = v;
    const int dxl = (x < 2) ? g.nx : 0;            // copy to x + nx
    const int dxr = (x >= g.nx - 2) ? -g.nx : 0;   // copy to x - nx
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

}  // namespace lbf

// Launchers implemented in the .cu files (host side).
namespace lbf {
cudaError_t launch_step(const StepArgs& a, int noise_mode, cudaStream_t s);
cudaError_t launch_noise49(float2* buf, const NoiseGenArgs& ga, const float2* twx, const float2* twy,
                           cudaStream_t s);
cudaError_t launch_stats_sample(const float* pops, const Grid& g, float2* z1, float2* z2,
                                const float2* twx, const float2* twy, double* bins, int nbins,
                                cudaStream_t s);
cudaError_t launch_bin_counts(int nx, int ny, int nbins, unsigned long long* counts, cudaStream_t s);
cudaError_t launch_fft2d(float2* data, int nx, int ny, int sign, const float2* twx, const float2* twy,
                         float scale, cudaStream_t s);
cudaError_t launch_set_plane(const double* src, float* plane, const Grid& g, int i, double fbar,
                             cudaStream_t s);
cudaError_t launch_get_plane(const float* plane, const Grid& g, int i, double fbar, double* out,
                             cudaStream_t s);
cudaError_t launch_moment(const float* pops, const Grid& g, int a, const double* fbar9, double* out,
                          cudaStream_t s);
cudaError_t launch_sums(const float* pops, const Grid& g, const double* fbar9, double* partial,
                        double* out3, cudaStream_t s);
int sums_partial_count();
}  // namespace lbf
