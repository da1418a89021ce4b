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
template <typename GA, typename C>
__device__ __forceinline__ void noise49_pair(const GA& ga, int mx, int my, C* zk, C* zmk) {
    using R = decltype(ga.a44);
    const uint32_t lin = (uint32_t)my * ga.nx + mx;
    const uint32_t cx = (uint32_t)((ga.nx - mx) & (ga.nx - 1));
    const uint32_t cy = (uint32_t)((ga.ny - my) & (ga.ny - 1));
    const uint32_t conj = cy * ga.nx + cx;
    const uint32_t owner = lin < conj ? lin : conj;
    const uint4 r = philox4x32_10(make_uint4(owner, ga.t_lo, ga.t_hi, TAG_KSPACE), ga.rk);
    R n0, n1, n2, n3;
    gauss_word(r.x, &n0, &n1);
    gauss_word(r.y, &n2, &n3);
    C e1, e2;
    if (lin == conj) {
        e1 = c_make(n0, R(0));
        e2 = c_make(n2, R(0));
    } else {
        const R h = R(0.70710678118654752440);
        e1 = c_make(n0 * h, n1 * h);
        e2 = c_make(n2 * h, n3 * h);
        if (lin != owner) { e1.y = -e1.y; e2.y = -e2.y; }
    }
    // Appendix B: k^2 = 10/3 - 4/3 (cos kx + cos ky) - 2/3 cos kx cos ky
    const R ckx = ga.cosx[mx], cky = ga.cosy[my];
    const R s = (R(10) / R(3)) - (R(4) / R(3)) * (ckx + cky) - (R(2) / R(3)) * (ckx * cky);
    const R x44 = ga.a44 + ga.b44 * s;
    const R x49 = ga.a49 + ga.b49 * s;
    const R x99 = ga.a99 + ga.b99 * s;
    R L44, L49, L94, L99;
    if (ga.eig) {
        // L = S diag(sqrt e1, sqrt e2), S = [[cos t, -sin t], [sin t, cos t]], t in [0, pi)
        // with tan 2t = 2 x49 / (x44 - x99), from the half-angle formulas (Sec. IV alternative)
        const R hm = R(0.5) * (x44 + x99), hd = R(0.5) * (x44 - x99);
        const R rad = sqrt(hd * hd + x49 * x49);
        const R ev1 = hm + rad, ev2 = fmax(hm - rad, R(0));
        const R c2t = rad > R(0) ? hd / rad : R(1);
        const R st = sqrt(fmax(R(0.5) * (R(1) - c2t), R(0)));
        const R ct = copysign(sqrt(fmax(R(0.5) * (R(1) + c2t), R(0))), x49 == R(0) ? R(1) : x49);
        const R r1 = sqrt(fmax(ev1, R(0))), r2 = sqrt(ev2);
        L44 = ct * r1; L49 = -st * r2; L94 = st * r1; L99 = ct * r2;
    } else {
        L44 = sqrt_fast(fmax(x44, R(0)));
        L49 = R(0);
        L94 = L44 > R(0) ? x49 * recip(L44) : R(0);
        L99 = sqrt_fast(fmax(x99 - L94 * L94, R(0)));
    }
    // xi_4(k) = L44 e1 + L49 e2, xi_9(k) = L94 e1 + L99 e2; at -k both are conjugated
    const C z4 = c_make(L44 * e1.x + L49 * e2.x, L44 * e1.y + L49 * e2.y);
    const C z9 = c_make(L94 * e1.x + L99 * e2.x, L94 * e1.y + L99 * e2.y);
    *zk = c_make(z4.x - z9.y, z4.y + z9.x);
    *zmk = c_make(z4.x + z9.y, -z4.y + z9.x);
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

// Position of H(k_x, y) in the column-permuted layout of the column pass: row y holds its
// nx values with the `count` columns of block b contiguous, element (y nx + b count + q),
// q the slot of k_x in paired_column.  A row pass gathers row y (one contiguous row) from it.
__device__ __forceinline__ long long perm_index(int x, int y, int nx, int count) {
    // count is a power of two: block b and slot of k_x = j (or nx - j) by shifts and masks
    const int half = count >> 1, hx = nx >> 1;
    const int lh = __ffs(half) - 1;
    const bool m = x > hx;
    const int j = m ? nx - x : x;              // 0 .. nx/2
    int p = ((j >> lh) << (lh + 1)) + (j & (half - 1)) + (m ? half : 0);    // b count + q
    if (x == hx) p = half;                     // block 0 pairs k_x = 0 (slot 0) with nx/2
    return (long long)y * nx + p;
}

// Correlated noise, first pass, for column block b: the CTA synthesises `count` k-space
// columns (half of them the mirrors of the others, so every (k, -k) draw is made once) for
// every k_y straight into shared memory (count * ny float2, padded), transforms them back
// along y and writes the partial result H(k_x, y) to out: PERM, in the column-permuted
// layout of perm_index (the block's count values of a row are one contiguous piece, a full
// 32-byte sector for count = 4, where the natural order splits them into two 16-byte pieces
// at k_x and -k_x), else row-major in place; a row pass finishes along x.
template <bool PERM, typename GA, typename C>
__device__ __forceinline__ void noise_cols_block(C* out, const GA& ga, int count, int b,
                                                 const C* __restrict__ twy) {
    extern __shared__ __align__(16) unsigned char noise_smem[];
    C* sm = reinterpret_cast<C*>(noise_smem);
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
            C z, zm;
            noise49_pair(ga, 0, ky, &z, &zm);
            sm[fpad(ky * count + 0)] = z;
            sm[fpad(kym * count + 0)] = zm;
            noise49_pair(ga, ga.nx >> 1, ky, &z, &zm);
            sm[fpad(ky * count + half)] = z;
            sm[fpad(kym * count + half)] = zm;
        } else {
            const int kym = (ny - ky) & (ny - 1);
            C z, zm;
            noise49_pair(ga, mx, ky, &z, &zm);
            sm[fpad(ky * count + q)] = z;
            sm[fpad(kym * count + q + half)] = zm;
        }
    }
    stockham_fft_out(sm, ny, log2n, count, -1, twy, [&](int e, C v) {
        const int q = e & (count - 1), y = e >> lc;
        out[(long long)y * ga.nx + (PERM ? b * count + q : paired_column(b, q, count, ga.nx))] = v;
    });
}

// Correlated noise, second pass, for row y: H(., y) gathered from the column-permuted layout
// src (written by noise_cols_block<true> with blocks of `count` columns), transformed back
// along x and scaled (the unitary n^-1/2), written to row y of dst (row-major).  One CTA per
// row with fft_threads(nx, 1) threads and fft_smem_bytes(nx, 1) of shared memory.
template <typename C, typename R>
__device__ __forceinline__ void noise_rows_gather(const C* __restrict__ src, C* __restrict__ dst, int nx, int count,
                                                  int y, const C* __restrict__ twx, R scale) {
    extern __shared__ __align__(16) unsigned char noise_smem[];
    C* sm = reinterpret_cast<C*>(noise_smem);
    C* rowp = dst + (long long)y * nx;
    const int log2n = 31 - __clz(nx);
    if (nx >= 256) {
        stockham_fft_io(sm, nx, log2n, 1, -1, twx, [&](int e) { return src[perm_index(e, y, nx, count)]; },
                        [&](int e, C v) { rowp[e] = c_make(v.x * scale, v.y * scale); });
        return;
    }
    for (int j = threadIdx.x; j < nx; j += blockDim.x) sm[fpad(j)] = src[perm_index(j, y, nx, count)];
    stockham_fft(sm, nx, log2n, 1, -1, twx);
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        const C v = sm[fpad(j)];
        rowp[j] = c_make(v.x * scale, v.y * scale);
    }
}

}  // namespace lbf
