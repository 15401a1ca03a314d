// Instantiations of the two-step plane kernels for one square plane side, FWI_N.
#include "launch.cuh"
#include "plane2.cuh"

namespace fwi {

template <int N>
void launch_plane2(int kind, dim3 g, size_t smem, cudaStream_t st, const StepParams& P) {
  if (kind == 0) k_plane2_mom<N, N><<<g, Plane2<N, N>::NT, smem, st>>>(P);
  else k_plane2_mass<N, N><<<g, Plane2<N, N>::NT, smem, st>>>(P);
}

template <int N>
void attrs_plane2(int cap) {
  set_smem_cap(k_plane2_mom<N, N>, cap);
  set_smem_cap(k_plane2_mass<N, N>, cap);
}

template void launch_plane2<FWI_N>(int, dim3, size_t, cudaStream_t, const StepParams&);
template void attrs_plane2<FWI_N>(int);

}  // namespace fwi
