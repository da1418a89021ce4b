// lb3d_q27.cu -- the D3Q27 step kernels (lb3d_kernel.cuh), in a translation unit of their own
// so that the two lattices compile in parallel.
#include "lb3d_kernel.cuh"

namespace lbf3 {

template cudaError_t launch_lattice<Lat27, float>(const Step3Args<float>&, const CUtensorMap*, const Launch3&,
                                                  cudaStream_t);
template cudaError_t launch_lattice<Lat27, double>(const Step3Args<double>&, const CUtensorMap*, const Launch3&,
                                                   cudaStream_t);

}  // namespace lbf3
