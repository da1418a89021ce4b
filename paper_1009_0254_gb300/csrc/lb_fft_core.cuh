// lb_fft_core.cuh -- in-place Stockham FFTs of power-of-two length in shared memory.
//
// `count` sequences of length n are interleaved element by element: element e of sequence
// c sits at s[pad(e * count + c)], with one float2 of padding after every 16 so that the
// strided accesses of every stage hit distinct banks.  A transform is a chain of Stockham
// stages (radix 16, then one radix 2/4/8 stage for the remaining factor); stage radix R with
// Ns = product of the previous radices maps, for work item j < n/R with k = j mod Ns,
//     a_m = s[j + m n/R] * W^(m k n/(Ns R)),   A = R-point DFT of a,
//     s[(j - k) R + k + m Ns] = A_m,
// which leaves the output in natural order.  W = exp(sign 2 pi i / n); sign = -1 is the
// e^{-i} kernel.  Each thread holds all values of its work items in registers between a
// read phase and a write phase separated by a barrier, so the stage runs in place.
#pragma once

#include <cuda_runtime.h>

namespace lbf {

__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_make(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 c_make(double x, double y) { return make_double2(x, y); }
// multiply by sign * i
template <typename C>
__device__ __forceinline__ C c_rot(C a, int sign) {
    return sign < 0 ? c_make(a.y, -a.x) : c_make(-a.y, a.x);
}

template <typename C>
__device__ __forceinline__ void dft2(C* a) {
    const C t = a[0];
    a[0] = c_add(t, a[1]);
    a[1] = c_sub(t, a[1]);
}

template <typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3, int sign) {
    const C y0 = c_add(a0, a2), y1 = c_sub(a0, a2);
    const C y2 = c_add(a1, a3), y3 = c_rot(c_sub(a1, a3), sign);
    a0 = c_add(y0, y2);
    a2 = c_sub(y0, y2);
    a1 = c_add(y1, y3);
    a3 = c_sub(y1, y3);
}

// 8-point DFT by decimation in time: X_k = E_k + W8^k O_k, X_{k+4} = E_k - W8^k O_k.
template <typename C>
__device__ __forceinline__ void dft8(C* a, int sign) {
    using R = decltype(a[0].x);
    C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4(e0, e1, e2, e3, sign);
    dft4(o0, o1, o2, o3, sign);
    const R h = R(0.70710678118654752440);
    const R s = (R)sign;
    o1 = c_mul(o1, c_make(h, s * h));
    o2 = c_rot(o2, sign);
    o3 = c_mul(o3, c_make(-h, s * h));
    a[0] = c_add(e0, o0); a[4] = c_sub(e0, o0);
    a[1] = c_add(e1, o1); a[5] = c_sub(e1, o1);
    a[2] = c_add(e2, o2); a[6] = c_sub(e2, o2);
    a[3] = c_add(e3, o3); a[7] = c_sub(e3, o3);
}

// 16-point DFT by decimation in time over two 8-point halves, W16^k = exp(sign i k pi / 8).
template <typename C>
__device__ __forceinline__ void dft16(C* a, int sign) {
    using R = decltype(a[0].x);
    C e[8], o[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        e[m] = a[2 * m];
        o[m] = a[2 * m + 1];
    }
    dft8(e, sign);
    dft8(o, sign);
    const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173), h = R(0.70710678118654752440);
    const R s = (R)sign;
    const C w[8] = {c_make(R(1), R(0)), c_make(c1, s * s1), c_make(h, s * h),
                    c_make(s1, s * c1), c_make(R(0), s),    c_make(-s1, s * c1),
                    c_make(-h, s * h),  c_make(-c1, s * s1)};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const C t = c_mul(o[k], w[k]);
        a[k] = c_add(e[k], t);
        a[k + 8] = c_sub(e[k], t);
    }
}

template <int R, typename C>
__device__ __forceinline__ void dft_r(C* a, int sign) {
    if (R == 2) dft2(a);
    else if (R == 4) dft4(a[0], a[1], a[2], a[3], sign);
    else if (R == 8) dft8(a, sign);
    else dft16(a, sign);
}

// One Stockham stage of radix R; each thread takes up to 16/R work items.  The twiddles
// W^(m t), m = 1 .. R-1, of a work item are running products of W^t (one table read per
// work item instead of R - 1; measured faster on the long transforms, and the products
// add ~1e-6 relative error in FP32).
template <int R, typename C>
__device__ __forceinline__ void stockham_stage(C* s, int n, int count, int lc, int Ns, int sign,
                                               const C* __restrict__ tw) {
    constexpr int MQ = 16 / R;
    const int items = (n / R) * count;
    const int T = blockDim.x;
    const int stride_in = n / R;
    const int tw_step = n / (Ns * R);
    C v[MQ][R];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int w = threadIdx.x + q * T;
        if (w < items) {
            const int c = w & (count - 1), j = w >> lc;
            const int k = j & (Ns - 1);
            using RT = decltype(tw[0].x);
            C t = Ns > 1 ? tw[k * tw_step] : c_make(RT(1), RT(0));
            if (sign > 0) t.y = -t.y;
            C wm = t;
#pragma unroll
            for (int m = 0; m < R; ++m) {
                C x = s[fpad((j + m * stride_in) * count + c)];
                if (m > 0 && Ns > 1) {
                    x = c_mul(x, wm);
                    if (m + 1 < R) wm = c_mul(wm, t);
                }
                v[q][m] = x;
            }
            dft_r<R>(v[q], sign);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int w = threadIdx.x + q * T;
        if (w < items) {
            const int c = w & (count - 1), j = w >> lc;
            const int k = j & (Ns - 1);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int m = 0; m < R; ++m) s[fpad((base + m * Ns) * count + c)] = v[q][m];
        }
    }
    __syncthreads();
}

// Full transform of `count` interleaved sequences of length n = 2^log2n (n >= 2) already in
// shared memory; tw[q] = exp(-2 pi i q / n), q < n.  Needs blockDim.x >= max(1, n/16) * count.
template <typename C>
__device__ __forceinline__ void stockham_fft(C* s, int n, int log2n, int count, int sign,
                                             const C* __restrict__ tw) {
    const int lc = 31 - __clz(count);
    int Ns = 1, left = log2n;
    __syncthreads();
    while (left >= 4) {
        stockham_stage<16>(s, n, count, lc, Ns, sign, tw);
        Ns <<= 4;
        left -= 4;
    }
    if (left == 3) stockham_stage<8>(s, n, count, lc, Ns, sign, tw);
    else if (left == 2) stockham_stage<4>(s, n, count, lc, Ns, sign, tw);
    else if (left == 1) stockham_stage<2>(s, n, count, lc, Ns, sign, tw);
}

// The same transform with its first stage reading the input through load(e) (e = element
// index * count + sequence) instead of from shared memory, and its last stage handing the
// output to store(e, value) instead of writing it back: two shared-memory passes fewer.
// Needs n >= 256 (a radix-16 first stage and at least one more); the shared buffer s is
// only a scratch between the stages.
template <int R, typename C, typename Load>
__device__ __forceinline__ void stockham_first(C* s, int n, int count, int lc, int sign, Load load) {
    constexpr int MQ = 16 / R;
    const int items = (n / R) * count;
    const int T = blockDim.x;
    const int stride_in = n / R;
    C v[MQ][R];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int w = threadIdx.x + q * T;
        if (w < items) {
            const int c = w & (count - 1), j = w >> lc;
#pragma unroll
            for (int m = 0; m < R; ++m) v[q][m] = load((j + m * stride_in) * count + c);
            dft_r<R>(v[q], sign);
        }
    }
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int w = threadIdx.x + q * T;
        if (w < items) {
            const int c = w & (count - 1), j = w >> lc;
#pragma unroll
            for (int m = 0; m < R; ++m) s[fpad((j * R + m) * count + c)] = v[q][m];
        }
    }
    __syncthreads();
}

template <int R, typename C, typename Store>
__device__ __forceinline__ void stockham_last(const C* s, int n, int count, int lc, int sign,
                                              const C* __restrict__ tw, Store store) {
    constexpr int MQ = 16 / R;
    const int Ns = n / R;            // last stage: Ns * R = n, so k = j and the output index is j + m Ns
    const int items = Ns * count;
    const int T = blockDim.x;
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int w = threadIdx.x + q * T;
        if (w < items) {
            const int c = w & (count - 1), j = w >> lc;
            C v[R];
            C t = tw[j];
            if (sign > 0) t.y = -t.y;
            C wm = t;
#pragma unroll
            for (int m = 0; m < R; ++m) {
                C x = s[fpad((j + m * Ns) * count + c)];
                if (m > 0) {
                    x = c_mul(x, wm);
                    if (m + 1 < R) wm = c_mul(wm, t);
                }
                v[m] = x;
            }
            dft_r<R>(v, sign);
#pragma unroll
            for (int m = 0; m < R; ++m) store((j + m * Ns) * count + c, v[m]);
        }
    }
}

template <typename C, typename Load, typename Store>
__device__ __forceinline__ void stockham_fft_io(C* s, int n, int log2n, int count, int sign,
                                                const C* __restrict__ tw, Load load, Store store) {
    const int lc = 31 - __clz(count);
    stockham_first<16>(s, n, count, lc, sign, load);
    int Ns = 16, left = log2n - 4;
    while (left > 4) {
        stockham_stage<16>(s, n, count, lc, Ns, sign, tw);
        Ns <<= 4;
        left -= 4;
    }
    if (left == 4) stockham_last<16>(s, n, count, lc, sign, tw, store);
    else if (left == 3) stockham_last<8>(s, n, count, lc, sign, tw, store);
    else if (left == 2) stockham_last<4>(s, n, count, lc, sign, tw, store);
    else stockham_last<2>(s, n, count, lc, sign, tw, store);
}

// Transform of sequences already in shared memory whose last stage hands the output to
// store(e, value) instead of writing it back (one shared-memory pass fewer).
template <typename C, typename Store>
__device__ __forceinline__ void stockham_fft_out(C* s, int n, int log2n, int count, int sign,
                                                 const C* __restrict__ tw, Store store) {
    const int lc = 31 - __clz(count);
    int Ns = 1, left = log2n;
    __syncthreads();
    while (left > 4) {
        stockham_stage<16>(s, n, count, lc, Ns, sign, tw);
        Ns <<= 4;
        left -= 4;
    }
    if (left == 4) stockham_last<16>(s, n, count, lc, sign, tw, store);
    else if (left == 3) stockham_last<8>(s, n, count, lc, sign, tw, store);
    else if (left == 2) stockham_last<4>(s, n, count, lc, sign, tw, store);
    else stockham_last<2>(s, n, count, lc, sign, tw, store);
}

__host__ __device__ inline int fft_threads(int n, int count) {
    int t = (n >= 16 ? n / 16 : 1) * count;
    if (t < 32) t = 32;
    return (t + 31) / 32 * 32;
}

__host__ __device__ inline size_t fft_smem_bytes(int n, int count, int elem_bytes = 8) {
    const long long e = (long long)n * count;
    return (size_t)(e + (e >> 4) + 1) * elem_bytes;
}

}  // namespace lbf
