// lb_spectra.cuh -- radial binning of the sampled spectra ([GACV] Sec. V A): the density
// structure factor S(k) = <|drho(k)|^2> and the longitudinal and transverse momentum spectra
// |k.j(k)|^2/|k|^2, |k x j(k)|^2/|k|^2, summed per radial bin of |k|.  Shared by the
// single-lattice sampler and the batched engine.
#pragma once

#include <cuda_runtime.h>

namespace lbf {

// Power of the three spectra at one wavevector k from Z1 = FT(drho + i jx) at k and -k and
// Z2 = FT(jy) at k, added to s[0..2].
__device__ __forceinline__ void add_power3(float2 a, float2 am, float2 c, float kx, float ky, float s[3]) {
    const float inv = rsqrtf(kx * kx + ky * ky);
    // two real fields in one transform: drho(k) = (Z(k) + Z(-k)*)/2, jx(k) = (Z(k) - Z(-k)*)/(2i)
    const float rr = 0.5f * (a.x + am.x), ri = 0.5f * (a.y - am.y);
    const float xr = 0.5f * (a.y + am.y), xi = -0.5f * (a.x - am.x);
    const float lr = (kx * xr + ky * c.x) * inv, li = (kx * xi + ky * c.y) * inv;
    const float tr = (-ky * xr + kx * c.x) * inv, ti = (-ky * xi + kx * c.y) * inv;
    s[0] += rr * rr + ri * ri;
    s[1] += lr * lr + li * li;
    s[2] += tr * tr + ti * ti;
}

// Adds the spectra of one nx x ny sample (power-of-two sides; z1, z2 its transforms; bin16
// the FP64-decided bin of every wavevector, 0xFFFF at k = 0) to the FP64 bins sb[3][nbins]
// in shared memory.  The bin depends on |k| only, so the up to four wavevectors (+-kx, +-ky)
// share it: the work is the half-plane mx <= nx/2, my <= ny/2, cut into units of one row and
// 32 consecutive mx, one unit per warp at a time (warp `gw` of `nw`), lanes along mx so the
// loads coalesce.  Each lane sums the powers of the distinct points of its set in FP32.
// Along a row the bin does not decrease with mx, so the lanes that share a bin are
// contiguous: a segmented warp reduction (FP32, at most 128 terms) leaves each run's sum in
// its first lane, which adds it to the FP64 bins.  Every lane of a warp must call this.
__device__ __forceinline__ void bin_half_plane(const float2* __restrict__ z1, const float2* __restrict__ z2,
                                               const unsigned short* __restrict__ bin16, int nx, int ny,
                                               int nbins, double* sb, int gw, int nw) {
    const int hx = nx / 2, hy = ny / 2;
    const int lane = threadIdx.x & 31;
    const int segs = (hx + 32) / 32;                 // units per row: mx = 0 .. hx
    const int units = (hy + 1) * segs;
    const float tpx = 6.2831853071795865f / (float)nx, tpy = 6.2831853071795865f / (float)ny;
    for (int u = gw; u < units; u += nw) {
        const int my = u / segs;
        const int mx = (u - my * segs) * 32 + lane;
        const int cy = (ny - my) & (ny - 1);
        const bool ypair = my != 0 && my != hy;      // -ky is another row
        const float ky = tpy * (float)my;
        const float kym = ypair ? -ky : ky;          // k_y of row cy (wrapped index)
        const long long r0 = (long long)my * nx, r1 = (long long)cy * nx;
        int b = -1;                                  // no bin: beyond nx/2, or k = 0
        float acc[3] = {0.f, 0.f, 0.f};
        if (mx <= hx) {
            const int bb = bin16[r0 + mx];
            if (bb != 0xFFFF) {
                b = bb;
                const int cx = (nx - mx) & (nx - 1);
                const bool xpair = mx != 0 && mx != hx;      // -kx is another column
                const float kx = tpx * (float)mx;
                const float kxm = xpair ? -kx : kx;
                const float2 A1 = z1[r0 + mx], A2 = z1[r1 + cx];
                add_power3(A1, A2, z2[r0 + mx], kx, ky, acc);                           // (mx, my)
                if (xpair || ypair) add_power3(A2, A1, z2[r1 + cx], kxm, kym, acc);     // (-mx, -my)
                if (xpair && ypair) {
                    const float2 A3 = z1[r0 + cx], A4 = z1[r1 + mx];
                    add_power3(A3, A4, z2[r0 + cx], kxm, ky, acc);                      // (-mx, my)
                    add_power3(A4, A3, z2[r1 + mx], kx, kym, acc);                      // (mx, -my)
                }
            }
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int bo = __shfl_down_sync(0xffffffffu, b, off);
            const float v0 = __shfl_down_sync(0xffffffffu, acc[0], off);
            const float v1 = __shfl_down_sync(0xffffffffu, acc[1], off);
            const float v2 = __shfl_down_sync(0xffffffffu, acc[2], off);
            if (lane + off < 32 && bo == b) {
                acc[0] += v0;
                acc[1] += v1;
                acc[2] += v2;
            }
        }
        const int bp = __shfl_up_sync(0xffffffffu, b, 1);
        if (b >= 0 && (lane == 0 || bp != b)) {
            atomicAdd(&sb[b], (double)acc[0]);
            atomicAdd(&sb[nbins + b], (double)acc[1]);
            atomicAdd(&sb[2 * nbins + b], (double)acc[2]);
        }
    }
}

}  // namespace lbf
