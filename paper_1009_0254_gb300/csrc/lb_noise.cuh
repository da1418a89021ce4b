// lb_noise.cuh -- k-space synthesis of the correlated noise of modes 4 and 9, [GACV]
// Sec. IV last paragraph: xi(k) = L(k) eta(k) with L L^T the (4,9) block of Xi(k),
// Eq. (noise-yeo), transformed back to the lattice with the unitary convention of Sec. III.
// Templated on the argument record (NoiseGenT with precomputed or on-the-fly Philox keys)
// so that the single-lattice path and the batched engine share it.
#pragma once

#include "lb_fft_core.cuh"
#include "lb_internal.cuh"

namespace lbf {

// Correlated noise of modes 4 and 9 in k-space: xi(k) = L(k) eta(k) with L L^T the
// (4,9) block of Xi(k), Eq. (noise-yeo); packed as Z = xi_4(k) + i xi_9(k).  The pair
// (k, -k) shares one Philox draw owned by the lower linear index, so eta(-k) = eta(k)*,
// and L(-k) = L(k).  noise49_pair returns Z(k) and Z(-k) from that one draw.
template <typename GA>
__device__ __forceinline__ void noise49_pair(const GA& ga, int mx, int my, float2* zk, float2* zmk) {
    const uint32_t lin = (uint32_t)my * ga.nx + mx;
    const uint32_t cx = (uint32_t)((ga.nx - mx) & (ga.nx - 1));
    const uint32_t cy = (uint32_t)((ga.ny - my) & (ga.ny - 1));
    const uint32_t conj = cy * ga.nx + cx;
    const uint32_t owner = lin < conj ? lin : conj;
    const uint4 r = philox4x32_10(make_uint4(owner, ga.t_lo, ga.t_hi, TAG_KSPACE), ga.rk);
    const float2 g01 = gauss_pair(r.x);
    const float2 g23 = gauss_pair(r.y);
    float2 e1, e2;
    if (lin == conj) {
        e1 = make_float2(g01.x, 0.f);
        e2 = make_float2(g23.x, 0.f);
    } else {
        const float h = 0.70710678118654752f;
        e1 = make_float2(g01.x * h, g01.y * h);
        e2 = make_float2(g23.x * h, g23.y * h);
        if (lin != owner) { e1.y = -e1.y; e2.y = -e2.y; }
    }
    // Appendix B: k^2 = 10/3 - 4/3 (cos kx + cos ky) - 2/3 cos kx cos ky
    const float ckx = ga.cosx[mx], cky = ga.cosy[my];
    const float s = (10.0f / 3.0f) - (4.0f / 3.0f) * (ckx + cky) - (2.0f / 3.0f) * (ckx * cky);
    const float x44 = ga.a44 + ga.b44 * s;
    const float x49 = ga.a49 + ga.b49 * s;
    const float x99 = ga.a99 + ga.b99 * s;
    float L44, L49, L94, L99;
    if (ga.eig) {
        // L = S diag(sqrt e1, sqrt e2), S = [[cos t, -sin t], [sin t, cos t]], t in [0, pi)
        // with tan 2t = 2 x49 / (x44 - x99), from the half-angle formulas (Sec. IV alternative)
        const float hm = 0.5f * (x44 + x99), hd = 0.5f * (x44 - x99);
        const float rad = sqrtf(hd * hd + x49 * x49);
        const float e1 = hm + rad, e2 = fmaxf(hm - rad, 0.f);
        const float c2t = rad > 0.f ? hd / rad : 1.f;
        const float st = sqrtf(fmaxf(0.5f * (1.f - c2t), 0.f));
        const float ct = copysignf(sqrtf(fmaxf(0.5f * (1.f + c2t), 0.f)), x49 == 0.f ? 1.f : x49);
        const float r1 = sqrtf(fmaxf(e1, 0.f)), r2 = sqrtf(e2);
        L44 = ct * r1; L49 = -st * r2; L94 = st * r1; L99 = ct * r2;
    } else {
        L44 = sqrt_approx(fmaxf(x44, 0.f));
        L49 = 0.f;
        L94 = L44 > 0.f ? x49 * rcp_approx(L44) : 0.f;
        L99 = sqrt_approx(fmaxf(x99 - L94 * L94, 0.f));
    }
    // xi_4(k) = L44 e1 + L49 e2, xi_9(k) = L94 e1 + L99 e2; at -k both are conjugated
    const float2 z4 = make_float2(L44 * e1.x + L49 * e2.x, L44 * e1.y + L49 * e2.y);
    const float2 z9 = make_float2(L94 * e1.x + L99 * e2.x, L94 * e1.y + L99 * e2.y);
    *zk = make_float2(z4.x - z9.y, z4.y + z9.x);
    *zmk = make_float2(z4.x + z9.y, -z4.y + z9.x);
}

// Columns handled by column-block b of width `count` (a power of two >= 2) in the paired
// synthesis: slot q < count/2 holds column j(b, q) of the left half and slot q + count/2
// its mirror nx - j (mod nx).  Block 0 pairs the self-mirrored columns 0 and nx/2.
__device__ __forceinline__ int paired_column(int b, int q, int count, int nx) {
    const int half = count >> 1;
    const int slot = q & (half - 1);
    const bool mirror = q >= half;
    if (b == 0 && slot == 0) return mirror ? nx >> 1 : 0;
    const int j = b * half + slot;                 // 1 .. nx/2 - 1
    return mirror ? nx - j : j;
}

// Correlated noise, first pass, for column block b: the CTA synthesises `count` k-space
// columns (half of them the mirrors of the others, so every (k, -k) draw is made once) for
// every k_y straight into shared memory (count * ny float2, padded), transforms them back
// along y and writes the partial result H(k_x, y) to out; a row pass finishes along x.
template <typename GA>
__device__ __forceinline__ void noise_cols_block(float2* out, const GA& ga, int count, int b,
                                                 const float2* __restrict__ twy) {
    extern __shared__ float2 sm[];
    const int ny = ga.ny, log2n = 31 - __clz(ny);
    const int lc = 31 - __clz(count);
    const int half = count >> 1;
    // owners: left slots q < half at every k_y; for the self-mirrored column pair of block 0
    // (columns 0 and nx/2) the partner of (k_x, k_y) is (k_x, -k_y) in the same column
    const int work = ny * half;
    for (int e = threadIdx.x; e < work; e += blockDim.x) {
        const int q = e & (half - 1), ky = e >> (lc - 1);
        const int mx = paired_column(b, q, count, ga.nx);
        if (b == 0 && q == 0) {
            // columns 0 and nx/2: draw for k_y <= ny/2, write k_y and ny - k_y of both
            if (ky > ny / 2) continue;
            const int kym = (ny - ky) & (ny - 1);
            float2 z, zm;
            noise49_pair(ga, 0, ky, &z, &zm);
            sm[fpad(ky * count + 0)] = z;
            sm[fpad(kym * count + 0)] = zm;
            noise49_pair(ga, ga.nx >> 1, ky, &z, &zm);
            sm[fpad(ky * count + half)] = z;
            sm[fpad(kym * count + half)] = zm;
        } else {
            const int kym = (ny - ky) & (ny - 1);
            float2 z, zm;
            noise49_pair(ga, mx, ky, &z, &zm);
            sm[fpad(ky * count + q)] = z;
            sm[fpad(kym * count + q + half)] = zm;
        }
    }
    stockham_fft(sm, ny, log2n, count, -1, twy);
    const int total = ny * count;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int q = e & (count - 1), y = e >> lc;
        out[(long long)y * ga.nx + paired_column(b, q, count, ga.nx)] = sm[fpad(e)];
    }
}

}  // namespace lbf
