// Instantiations of the two-step z pass for one z length, FWI_N (both tiles, both modes).
#include "launch.cuh"
#include "plane2.cuh"

namespace fwi {

template <int NZ>
void launch_zpass2(int mode, int tz, dim3 g, size_t smem, cudaStream_t st, const StepParams& P) {
  if (tz == 32) {
    if (mode == 0) k_zpass2<0, NZ, 32><<<g, Z2<NZ, 32>::NT, smem, st>>>(P);
    else k_zpass2<1, NZ, 32><<<g, Z2<NZ, 32>::NT, smem, st>>>(P);
  } else {
    if (mode == 0) k_zpass2<0, NZ, 16><<<g, Z2<NZ, 16>::NT, smem, st>>>(P);
    else k_zpass2<1, NZ, 16><<<g, Z2<NZ, 16>::NT, smem, st>>>(P);
  }
}

template <int NZ>
void attrs_zpass2(int cap) {
  set_smem_cap(k_zpass2<0, NZ, 32>, cap);
  set_smem_cap(k_zpass2<1, NZ, 32>, cap);
  set_smem_cap(k_zpass2<0, NZ, 16>, cap);
  set_smem_cap(k_zpass2<1, NZ, 16>, cap);
}

template void launch_zpass2<FWI_N>(int, int, dim3, size_t, cudaStream_t, const StepParams&);
template void attrs_zpass2<FWI_N>(int);

}  // namespace fwi
