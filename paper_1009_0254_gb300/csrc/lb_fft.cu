// lb_fft.cu -- power-of-two FFTs in shared memory, the k-space synthesis of the correlated
// noise ([GACV] Sec. IV, last paragraph) and the sampled spectra ([GACV] Sec. V A).
//
// Transforms follow the unitary convention of [GACV] Sec. III:
//   forward  a(k) = n^-1/2 sum_r exp(+i k.r) a(r)         (sign = +1)
//   back     a(r) = n^-1/2 sum_k exp(-i k.r) a(k)         (sign = -1)
// with k = 2 pi (mx/nx, my/ny).  Sizes are powers of two.  Each transform is a 2D
// pass over rows (one CTA per row) and a pass over columns (a CTA per strip of C
// adjacent columns), each an in-place Stockham FFT in shared memory (lb_fft_core.cuh)
// with a twiddle table exp(-2 pi i q/n) computed on the host in FP64 (one read per
// butterfly, its powers formed on the fly).
#include <algorithm>

#include "lb_fft_core.cuh"
#include "lb_internal.cuh"
#include "lb_noise.cuh"
#include "lb_spectra.cuh"

namespace lbf {

__device__ __forceinline__ int ilog2(int n) { return 31 - __clz(n); }

// Row pass, in place, scaled by `scale` on the way out.  One CTA per row; rows of 256 and
// more points read and write global memory in the first and last stage directly.
__global__ void __launch_bounds__(1024) fft_rows_kernel(float2* data, int nx, int sign, const float2* __restrict__ twx, float scale) {
    extern __shared__ float2 sm[];
    const int log2n = ilog2(nx);
    float2* rowp = data + (long long)blockIdx.x * nx;
    if (nx >= 256) {
        stockham_fft_io(sm, nx, log2n, 1, sign, twx, [&](int e) { return rowp[e]; },
                        [&](int e, float2 v) { rowp[e] = make_float2(v.x * scale, v.y * scale); });
        return;
    }
    for (int j = threadIdx.x; j < nx; j += blockDim.x) sm[fpad(j)] = rowp[j];
    stockham_fft(sm, nx, log2n, 1, sign, twx);
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        const float2 v = sm[fpad(j)];
        rowp[j] = make_float2(v.x * scale, v.y * scale);
    }
}

// Correlated noise, first pass (lb_noise.cuh noise_cols_block): one CTA per block of
// `count` k-space columns.  PERM: written column-permuted to a scratch field, from which the
// second pass gathers every row and transforms it along x into the noise field; else in
// place, finished by the plain row pass.
template <bool PERM>
__global__ void __launch_bounds__(1024) noise_cols_kernel(float2* out, NoiseGenArgs ga, int count,
                                                          const float2* __restrict__ twy) {
    noise_cols_block<PERM>(out, ga, count, blockIdx.x, twy);
}

__global__ void __launch_bounds__(1024) noise_rows_kernel(const float2* __restrict__ h, float2* xi, int nx, int ny,
                                                          int count, const float2* __restrict__ twx, float scale) {
    noise_rows_gather(h, xi, nx, count, (int)blockIdx.x, twx, scale);
}

// FP64 storage: the same two passes of the correlated noise in FP64 (rows: one CTA per row).
__global__ void __launch_bounds__(512) fft_rows_kernel_d(double2* data, int nx, int sign,
                                                          const double2* __restrict__ twx, double scale) {
    extern __shared__ __align__(16) unsigned char rows_smem_d[];
    double2* sm = reinterpret_cast<double2*>(rows_smem_d);
    double2* rowp = data + (long long)blockIdx.x * nx;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) sm[fpad(j)] = rowp[j];
    stockham_fft(sm, nx, ilog2(nx), 1, sign, twx);
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        const double2 v = sm[fpad(j)];
        rowp[j] = make_double2(v.x * scale, v.y * scale);
    }
}

__global__ void __launch_bounds__(512) noise_cols_kernel_d(double2* out, NoiseGenArgsD ga, int count,
                                                            const double2* __restrict__ twy) {
    noise_cols_block<false>(out, ga, count, blockIdx.x, twy);
}

// Column pass over strips of `count` adjacent columns, scaled by `scale` on the way out.
__global__ void __launch_bounds__(1024) fft_cols_kernel(float2* data, int nx, int ny, int count, int sign,
                                const float2* __restrict__ twy, float scale) {
    extern __shared__ float2 sm[];
    const int log2n = ilog2(ny);
    const int xs = blockIdx.x * count;
    const int total = ny * count;
    const int lc = 31 - __clz(count);
    constexpr int U = 8;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = e < total ? data[(long long)(e >> lc) * nx + xs + (e & (count - 1))] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < total) sm[fpad(e)] = v[u];
        }
    }
    stockham_fft(sm, ny, log2n, count, sign, twy);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const float2 v = sm[fpad(e)];
        data[(long long)(e >> lc) * nx + xs + (e & (count - 1))] = make_float2(v.x * scale, v.y * scale);
    }
}

static int col_strip(int nx, int ny) {
    // strip width: as many columns as fit in one CTA (<= 1024 threads, ~200 KB), at most 16
    int c = 16;
    while (c > 1 && (fft_threads(ny, c) > 1024 || fft_smem_bytes(ny, c) > 200 * 1024)) c >>= 1;
    if (c > nx) c = nx;
    return c;
}

static cudaError_t rows_pass(float2* data, int nx, int ny, int sign, const float2* twx, float scale,
                             cudaStream_t s) {
    const size_t smem = fft_smem_bytes(nx, 1);
    cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fft_rows_kernel<<<ny, fft_threads(nx, 1), smem, s>>>(data, nx, sign, twx, scale);
    return cudaGetLastError();
}

static cudaError_t cols_pass(float2* data, int nx, int ny, int sign, const float2* twy, float scale,
                             cudaStream_t s) {
    const int c = col_strip(nx, ny);
    const size_t smem = fft_smem_bytes(ny, c);
    cudaError_t e = cudaFuncSetAttribute(fft_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fft_cols_kernel<<<nx / c, fft_threads(ny, c), smem, s>>>(data, nx, ny, c, sign, twy, scale);
    return cudaGetLastError();
}

cudaError_t launch_fft2d(float2* data, int nx, int ny, int sign, const float2* twx, const float2* twy,
                         float scale, cudaStream_t s) {
    cudaError_t e = rows_pass(data, nx, ny, sign, twx, 1.0f, s);
    if (e != cudaSuccess) return e;
    return cols_pass(data, nx, ny, sign, twy, scale, s);
}

cudaError_t launch_noise49(float2* buf, float2* scratch, const NoiseGenArgs& ga, const float2* twx,
                           const float2* twy, cudaStream_t s) {
    // synthesise xi(k) column block by column block and transform back along y, then along
    // x with the unitary n^-1/2 into buf; the paired blocks need an even width (ny <= 8192).
    // Rows of 256 points and more go through the column-permuted scratch (whole 32-byte
    // sectors per write, rows gathered back in the first stage of the row transform:
    // 219 -> 171 us at 4096^2, 118 -> 115 us a step at 2048^2); shorter rows stay in place.
    const int c = col_strip(ga.nx, ga.ny);
    if (c < 2) return cudaErrorInvalidValue;
    const bool perm = ga.nx >= 256;
    const size_t smem = fft_smem_bytes(ga.ny, c);
    const float scale = (float)(1.0 / sqrt((double)ga.nx * (double)ga.ny));
    cudaError_t e;
    if (!perm) {
        e = cudaFuncSetAttribute(noise_cols_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        noise_cols_kernel<false><<<ga.nx / c, fft_threads(ga.ny, c), smem, s>>>(buf, ga, c, twy);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return rows_pass(buf, ga.nx, ga.ny, -1, twx, scale, s);
    }
    e = cudaFuncSetAttribute(noise_cols_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    noise_cols_kernel<true><<<ga.nx / c, fft_threads(ga.ny, c), smem, s>>>(scratch, ga, c, twy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t rsm = fft_smem_bytes(ga.nx, 1);
    e = cudaFuncSetAttribute(noise_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    if (e != cudaSuccess) return e;
    noise_rows_kernel<<<ga.ny, fft_threads(ga.nx, 1), rsm, s>>>(scratch, buf, ga.nx, ga.ny, c, twx, scale);
    return cudaGetLastError();
}

int noise_strip_d(int nx, int ny) {
    int c = 16;
    while (c > 1 && (fft_threads(ny, c) > 512 || fft_smem_bytes(ny, c, 16) > 200 * 1024)) c >>= 1;
    return c > nx ? nx : c;
}

cudaError_t launch_noise49_d(double2* buf, const NoiseGenArgsD& ga, const double2* twx, const double2* twy,
                             cudaStream_t s) {
    const int c = noise_strip_d(ga.nx, ga.ny);
    if (c < 2) return cudaErrorInvalidValue;
    const size_t smem = fft_smem_bytes(ga.ny, c, 16);
    cudaError_t e = cudaFuncSetAttribute(noise_cols_kernel_d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    noise_cols_kernel_d<<<ga.nx / c, fft_threads(ga.ny, c), smem, s>>>(buf, ga, c, twy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t rsm = fft_smem_bytes(ga.nx, 1, 16);
    e = cudaFuncSetAttribute(fft_rows_kernel_d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    if (e != cudaSuccess) return e;
    fft_rows_kernel_d<<<ga.ny, fft_threads(ga.nx, 1), rsm, s>>>(buf, ga.nx, -1, twx,
                                                                1.0 / sqrt((double)ga.nx * (double)ga.ny));
    return cudaGetLastError();
}

// --- sampled spectra ---------------------------------------------------------------

// z1 = drho + i jx, z2 = jy of the pre-collision state f_i(r) = f*_i(r - c_i)
template <typename T>
__global__ void stats_fields_kernel(const T* __restrict__ src, Grid g, float2* z1, float2* z2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.nx) return;
    const long long P = g.plane;
    const long long c = g.at(x, y);
    const float f0 = Elem<T>::load(src[c], 0), f1 = Elem<T>::load(src[P + c - 1], 1);
    const float f2 = Elem<T>::load(src[2 * P + c - g.pitch], 2), f3 = Elem<T>::load(src[3 * P + c + 1], 3);
    const float f4 = Elem<T>::load(src[4 * P + c + g.pitch], 4), f5 = Elem<T>::load(src[5 * P + c - g.pitch - 1], 5);
    const float f6 = Elem<T>::load(src[6 * P + c - g.pitch + 1], 6), f7 = Elem<T>::load(src[7 * P + c + g.pitch + 1], 7);
    const float f8 = Elem<T>::load(src[8 * P + c + g.pitch - 1], 8);
    const float drho = f0 + ((f1 + f3) + (f2 + f4)) + ((f5 + f7) + (f6 + f8));
    const float jx = (f1 - f3) + (f5 - f7) + (f8 - f6);
    const float jy = (f2 - f4) + (f5 - f7) + (f6 - f8);
    const long long o = (long long)y * g.nx + x;
    z1[o] = make_float2(drho, jx);
    z2[o] = make_float2(jy, 0.f);
}

// Radial bin of wavevector (mx, my), decided in FP64 with explicitly rounded
// operations (no contraction), matching a plain double evaluation of
// floor(sqrt(kx^2 + ky^2) / (pi sqrt 2 / nbins)), kx = (2 pi mx_w) / nx.
__device__ __forceinline__ int k_bin(int mx, int my, int nx, int ny, int nbins, double* kx_o, double* ky_o) {
    const int mxw = mx > nx / 2 ? mx - nx : mx;
    const int myw = my > ny / 2 ? my - ny : my;
    const double two_pi = 6.283185307179586;
    const double kx = __ddiv_rn(__dmul_rn(two_pi, (double)mxw), (double)nx);
    const double ky = __ddiv_rn(__dmul_rn(two_pi, (double)myw), (double)ny);
    const double km = __dsqrt_rn(__dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky)));
    const double width = __ddiv_rn(__dmul_rn(3.141592653589793, 1.4142135623730951), (double)nbins);
    int b = (int)floor(__ddiv_rn(km, width));
    if (b > nbins - 1) b = nbins - 1;
    *kx_o = kx;
    *ky_o = ky;
    return b;
}

// Radial spectra of one sample (lb_spectra.cuh): the block's warps share the half-plane
// units, the block's FP64 bins in shared memory are added to the global bins at the end.
__global__ void bin_kernel(const float2* __restrict__ z1, const float2* __restrict__ z2,
                           const unsigned short* __restrict__ bin16, int nx, int ny, int nbins, double* bins) {
    extern __shared__ double sb[];   // 3 * nbins
    for (int j = threadIdx.x; j < 3 * nbins; j += blockDim.x) sb[j] = 0.0;
    __syncthreads();
    const int wpb = blockDim.x >> 5;
    bin_half_plane(z1, z2, bin16, nx, ny, nbins, sb, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb);
    __syncthreads();
    for (int j = threadIdx.x; j < 3 * nbins; j += blockDim.x)
        if (sb[j] != 0.0) atomicAdd(&bins[j], sb[j]);
}

// Bin of every wavevector (0xFFFF for k = 0) and the bin counts, decided in FP64 once.
__global__ void bin_table_kernel(int nx, int ny, int nbins, unsigned short* bin16, unsigned long long* counts) {
    const long long n = (long long)nx * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (i == 0) {
            bin16[0] = 0xFFFF;
            continue;
        }
        double kx, ky;
        const int b = k_bin((int)(i % nx), (int)(i / nx), nx, ny, nbins, &kx, &ky);
        bin16[i] = (unsigned short)b;
        atomicAdd(&counts[b], 1ull);
    }
}

cudaError_t launch_bin_counts(int nx, int ny, int nbins, unsigned short* bin16, unsigned long long* counts,
                              cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * nbins, s);
    if (e != cudaSuccess) return e;
    bin_table_kernel<<<1024, 256, 0, s>>>(nx, ny, nbins, bin16, counts);
    return cudaGetLastError();
}

cudaError_t launch_stats_sample(const void* pops, int storage, const Grid& g, float2* z1, float2* z2,
                                const float2* twx, const float2* twy, const unsigned short* bin16, double* bins,
                                int nbins, cudaStream_t s) {
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny);
    if (storage == 1) stats_fields_kernel<__half><<<grd, blk, 0, s>>>(static_cast<const __half*>(pops), g, z1, z2);
    else if (storage == 2) stats_fields_kernel<double><<<grd, blk, 0, s>>>(static_cast<const double*>(pops), g, z1, z2);
    else stats_fields_kernel<float><<<grd, blk, 0, s>>>(static_cast<const float*>(pops), g, z1, z2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float scale = (float)(1.0 / sqrt((double)g.nx * (double)g.ny));
    e = launch_fft2d(z1, g.nx, g.ny, +1, twx, twy, scale, s);
    if (e != cudaSuccess) return e;
    e = launch_fft2d(z2, g.nx, g.ny, +1, twx, twy, scale, s);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)3 * nbins * sizeof(double);
    e = cudaFuncSetAttribute(bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long units = (long long)(g.ny / 2 + 1) * ((g.nx / 2 + 32) / 32);   // warp work units
    const int nblk = (int)std::min<long long>(304, std::max<long long>(1, units / 32));   // <= 2 per SM
    bin_kernel<<<nblk, 256, smem, s>>>(z1, z2, bin16, g.nx, g.ny, nbins, bins);
    return cudaGetLastError();
}

}  // namespace lbf
