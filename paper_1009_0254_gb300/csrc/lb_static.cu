// lb_static.cu -- conserved sums of caller-owned populations without any device
// allocation: the block partial sums live in a file-scope __device__ array.
//
// This exists for callers that cannot call cudaMalloc: code whose device memory is
// entirely owned by another allocator (a host framework that has reserved the GPU's
// memory for its own pool), or latency-critical loops that must not trigger the
// implicit device-wide synchronisation a cudaMalloc/cudaFree pair can cause.  They pass
// device pointers to their populations and to a 3-double result and get the same FP64
// sums as lb_moments, computed in a fixed order (deterministic for a given size).
#include <mutex>
#include <string>

#include "lb_internal.cuh"
#include "lbfluct.h"

// The scratch: one FP64 triple {rho, jx, jy} per lattice row, LB_STATIC_MAX_ROWS rows
// (384 KB), resident on every device that loads the library until the process exits.
// Every call writes the rows it uses before reading them; rows beyond the current ny
// keep an earlier call's values and are never read.
static __device__ __align__(256) double g_row_sums[LB_STATIC_MAX_ROWS * 3];

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

__constant__ int kCXs[lbf::Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCYs[lbf::Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Host-side address of g_row_sums on each device, looked up once per device.
double* g_row_sums_addr[kMaxDevices] = {nullptr};
std::mutex g_addr_mutex;

__global__ void row_sums_kernel(const double* __restrict__ f, int nx, int ny, double* __restrict__ rows) {
    __shared__ double sh[3][kThreads];
    const int y = blockIdx.x;
    const long long n = (long long)nx * ny;
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int x = threadIdx.x; x < nx; x += kThreads) {
        const long long s = (long long)y * nx + x;
#pragma unroll
        for (int i = 0; i < lbf::Q; ++i) {
            const double v = f[i * n + s];
            r += v;
            jx += kCXs[i] * v;
            jy += kCYs[i] * v;
        }
    }
    sh[0][threadIdx.x] = r;
    sh[1][threadIdx.x] = jx;
    sh[2][threadIdx.x] = jy;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) rows[3 * y + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void total_kernel(const double* __restrict__ rows, int ny, double* __restrict__ out) {
    __shared__ double sh[3][kThreads];
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int y = threadIdx.x; y < ny; y += kThreads) s += rows[3 * y + c];
        sh[c][threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = sh[threadIdx.x][0];
}

int fail_static(int code, const std::string& msg) {
    lbf::set_context_free_error(msg);     // reported by lb_last_error(NULL)
    return code;
}

}  // namespace

extern "C" int lb_conserved_sums_static(const double* f, int nx, int ny, double* sums, void* stream) {
    if (!f || !sums) return fail_static(LB_EINVAL, "f and sums must be device pointers");
    if (nx < 1 || ny < 1) return fail_static(LB_EINVAL, "nx and ny must be >= 1");
    if (ny > LB_STATIC_MAX_ROWS)
        return fail_static(LB_EINVAL, "ny exceeds LB_STATIC_MAX_ROWS (" + std::to_string(LB_STATIC_MAX_ROWS) +
                                          "), the row capacity of the static scratch array");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_static(LB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_static(LB_EINVAL, "device ordinal out of range");
    double* rows = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_addr_mutex);
        if (!g_row_sums_addr[dev]) {
            // once per device, with that device current: the device address of the array
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_row_sums);
            if (e != cudaSuccess)
                return fail_static(LB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_row_sums_addr[dev] = static_cast<double*>(p);
        }
        rows = g_row_sums_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    row_sums_kernel<<<ny, kThreads, 0, s>>>(f, nx, ny, rows);
    total_kernel<<<1, kThreads, 0, s>>>(rows, ny, sums);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_static(LB_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return LB_OK;
}
