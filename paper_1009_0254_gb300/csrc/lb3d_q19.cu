// lb3d_q19.cu -- the D3Q19 step kernels (lb3d_kernel.cuh), in a translation unit of their own
// so that the two lattices compile in parallel.
#include "lb3d_kernel.cuh"

namespace lbf3 {

template cudaError_t launch_lattice<Lat19, float>(const Step3Args<float>&, const CUtensorMap*, const Launch3&,
                                                  cudaStream_t);
template cudaError_t launch_lattice<Lat19, double>(const Step3Args<double>&, const CUtensorMap*, const Launch3&,
                                                   cudaStream_t);

}  // namespace lbf3
