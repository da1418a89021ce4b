// lb_io.cu -- conversion between the ABI's FP64 pre-collision populations and the
// stored FP32 post-collision deviations, FP64 moments and the FP64 conserved sums.
//
// Stored plane i holds df*_i(r) = f*_i(r, t-1) - fbar_i; the pre-collision state is
// f_i(r, t) = fbar_i + df*_i(r - c_i), so writing a state f_i(r) stores
// df*_i(r) = f_i(r + c_i) - fbar_i (periodic).
#include "lb_internal.cuh"

namespace lbf {

__constant__ int kCX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
// rows of T, [GACV] Table I / Eq. (Tmat)
__constant__ double kTm[Q][Q] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {-2, 1, 1, 1, 1, 4, 4, 4, 4},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, -1, 0, 1, 0, 2, -2, -2, 2},
    {0, 0, -1, 0, 1, 2, 2, -2, -2},
    {2, -4, -4, -4, -4, 8, 8, 8, 8}};

template <typename T>
__global__ void set_plane_kernel(const double* __restrict__ src, T* plane, Grid g, int i, double fbar) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.nx) return;
    int xs = x + kCX[i], ys = y + kCY[i];
    xs = xs < 0 ? xs + g.nx : (xs >= g.nx ? xs - g.nx : xs);
    ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
    const double v = src[(long long)ys * g.nx + xs] - fbar;
    store_with_ghosts(plane, g, x, y, Elem<T>::store((typename Arith<T>::type)v, i));
}

template <typename T>
__global__ void get_plane_kernel(const T* __restrict__ plane, Grid g, int i, double fbar, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.nx) return;
    out[(long long)y * g.nx + x] = fbar + (double)Elem<T>::load(plane[g.at(x - kCX[i], y - kCY[i])], i);
}

template <typename T>
__device__ __forceinline__ void pulled_f64(const T* __restrict__ pops, const Grid& g, int x, int y,
                                           const double* fbar9, double f[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
        f[i] = fbar9[i] + (double)Elem<T>::load(pops[i * g.plane + g.at(x - kCX[i], y - kCY[i])], i);
}

template <typename T>
__global__ void moment_kernel(const T* __restrict__ pops, Grid g, int a, const double* __restrict__ fbar9,
                              double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.nx) return;
    double f[Q];
    pulled_f64(pops, g, x, y, fbar9, f);
    double m = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) m += kTm[a][i] * f[i];
    out[(long long)y * g.nx + x] = m;
}

constexpr int SUM_BLOCKS = 512;
constexpr int SUM_THREADS = 256;
int sums_partial_count() { return SUM_BLOCKS * 3; }

// FP64 sums of rho, jx, jy in a fixed order: per-thread strided sums, a block tree,
// then one block over the partials (deterministic for a given lattice size).
template <typename T>
__global__ void sums_kernel(const T* __restrict__ pops, Grid g, const double* __restrict__ fbar9,
                            double* partial) {
    __shared__ double sh[3][SUM_THREADS];
    double s0 = 0, s1 = 0, s2 = 0;
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)SUM_THREADS + threadIdx.x; k < n;
         k += (long long)SUM_BLOCKS * SUM_THREADS) {
        const int x = (int)(k % g.nx), y = (int)(k / g.nx);
        double f[Q];
        pulled_f64(pops, g, x, y, fbar9, f);
        double r = 0, jx = 0, jy = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            r += f[i];
            jx += kTm[1][i] * f[i];
            jy += kTm[2][i] * f[i];
        }
        s0 += r; s1 += jx; s2 += jy;
    }
    sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = s1; sh[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = SUM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) partial[blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void sums_final_kernel(const double* __restrict__ partial, double* out3) {
    __shared__ double sh[3][SUM_THREADS];
    for (int c = 0; c < 3; ++c) {
        double s = 0;
        for (int b = threadIdx.x; b < SUM_BLOCKS; b += SUM_THREADS) s += partial[b * 3 + c];
        sh[c][threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = SUM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) out3[threadIdx.x] = sh[threadIdx.x][0];
}

static dim3 row_grid(const Grid& g, int bx) { return dim3((g.nx + bx - 1) / bx, g.ny); }

// `storage`: 0 FP32, 1 FP16 deviations, 2 FP64 (the LB_FP32 / LB_FP16DEV / LB_FP64 codes)
cudaError_t launch_set_plane(const double* src, void* pops, int storage, const Grid& g, int i, double fbar,
                             cudaStream_t s) {
    if (storage == 1)
        set_plane_kernel<__half><<<row_grid(g, 128), 128, 0, s>>>(src, static_cast<__half*>(pops) + i * g.plane, g, i, fbar);
    else if (storage == 2)
        set_plane_kernel<double><<<row_grid(g, 128), 128, 0, s>>>(src, static_cast<double*>(pops) + i * g.plane, g, i, fbar);
    else
        set_plane_kernel<float><<<row_grid(g, 128), 128, 0, s>>>(src, static_cast<float*>(pops) + i * g.plane, g, i, fbar);
    return cudaGetLastError();
}

cudaError_t launch_get_plane(const void* pops, int storage, const Grid& g, int i, double fbar, double* out,
                             cudaStream_t s) {
    if (storage == 1)
        get_plane_kernel<__half><<<row_grid(g, 128), 128, 0, s>>>(static_cast<const __half*>(pops) + i * g.plane, g, i,
                                                                 fbar, out);
    else if (storage == 2)
        get_plane_kernel<double><<<row_grid(g, 128), 128, 0, s>>>(static_cast<const double*>(pops) + i * g.plane, g, i,
                                                                 fbar, out);
    else
        get_plane_kernel<float><<<row_grid(g, 128), 128, 0, s>>>(static_cast<const float*>(pops) + i * g.plane, g, i,
                                                                fbar, out);
    return cudaGetLastError();
}

cudaError_t launch_moment(const void* pops, int storage, const Grid& g, int a, const double* fbar9, double* out,
                          cudaStream_t s) {
    if (storage == 1)
        moment_kernel<__half><<<row_grid(g, 128), 128, 0, s>>>(static_cast<const __half*>(pops), g, a, fbar9, out);
    else if (storage == 2)
        moment_kernel<double><<<row_grid(g, 128), 128, 0, s>>>(static_cast<const double*>(pops), g, a, fbar9, out);
    else
        moment_kernel<float><<<row_grid(g, 128), 128, 0, s>>>(static_cast<const float*>(pops), g, a, fbar9, out);
    return cudaGetLastError();
}

cudaError_t launch_sums(const void* pops, int storage, const Grid& g, const double* fbar9, double* partial, double* out3,
                        cudaStream_t s) {
    if (storage == 1)
        sums_kernel<__half><<<SUM_BLOCKS, SUM_THREADS, 0, s>>>(static_cast<const __half*>(pops), g, fbar9, partial);
    else if (storage == 2)
        sums_kernel<double><<<SUM_BLOCKS, SUM_THREADS, 0, s>>>(static_cast<const double*>(pops), g, fbar9, partial);
    else
        sums_kernel<float><<<SUM_BLOCKS, SUM_THREADS, 0, s>>>(static_cast<const float*>(pops), g, fbar9, partial);
    sums_final_kernel<<<1, SUM_THREADS, 0, s>>>(partial, out3);
    return cudaGetLastError();
}

}  // namespace lbf
