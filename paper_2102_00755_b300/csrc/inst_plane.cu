// Instantiations of the warp-owned plane kernels for one square plane side FWI_N
// (0: runtime radix schedules) with FWI_E values staged per lane.
#include "launch.cuh"

namespace fwi {

template <int E, int F>
void launch_plane(int kind, dim3 g, size_t smem, cudaStream_t st, const StepParams& P) {
  if (kind == 0) k_plane_mom<E, F, F><<<g, kTpbPlane, smem, st>>>(P);
  else if (kind == 1) k_plane_mass<E, F, F><<<g, kTpbPlane, smem, st>>>(P);
  else k_tr_init<E, F, F><<<g, kTpbPlane, smem, st>>>(P);
}

template <int E, int F>
void attrs_plane(int cap) {
  set_smem_cap(k_plane_mom<E, F, F>, cap);
  set_smem_cap(k_plane_mass<E, F, F>, cap);
  set_smem_cap(k_tr_init<E, F, F>, cap);
}

template void launch_plane<FWI_E, FWI_N>(int, dim3, size_t, cudaStream_t, const StepParams&);
template void attrs_plane<FWI_E, FWI_N>(int);

}  // namespace fwi
