// lb_selftest.cu -- exercises the device-side timeout path of the TMA step kernels without
// any fault: one CTA arms an mbarrier for a transfer that is never issued and waits on it
// with the same bounded wait the kernels use; the wait gives up after the limit and the
// kernel reports it, leaving the context usable.
#include "lb_tma.cuh"
#include "lbfluct.h"

namespace lbf {

__global__ void bounded_wait_probe_kernel(unsigned long long limit_ns, int* gave_up) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(smem_u32(&bar), 16);   // 16 bytes that never arrive
    const bool ok = mbar_wait_bounded_ns(smem_u32(&bar), 0, limit_ns);
    const int any = __syncthreads_or(!ok);
    if (threadIdx.x == 0) *gave_up = any;
}

}  // namespace lbf

extern "C" int lb_selftest_bounded_wait(double limit_s, int* gave_up) {
    if (!(limit_s > 0.0) || limit_s > 10.0) return LB_EINVAL;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return LB_ENOMEM;
    int h = -1;
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        lbf::bounded_wait_probe_kernel<<<1, 64>>>((unsigned long long)(limit_s * 1e9), d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return LB_ECUDA;
    if (gave_up) *gave_up = h;
    return h == 1 ? LB_ETIMEOUT : (h == 0 ? LB_OK : LB_ECUDA);
}
