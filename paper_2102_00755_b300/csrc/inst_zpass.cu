// Instantiations of the warp-owned z pass for one length FWI_N (0: runtime radix
// schedule) with FWI_E values staged per lane (both tiles, both modes).
#include "launch.cuh"

namespace fwi {

template <int E, int FZ>
void launch_zpass(int mode, int tz, dim3 g, size_t smem, cudaStream_t st, const StepParams& P) {
  if (tz == 32) {
    if (mode == 0) k_zpass<0, E, FZ, 32><<<g, kTpbZ, smem, st>>>(P);
    else k_zpass<1, E, FZ, 32><<<g, kTpbZ, smem, st>>>(P);
  } else {
    if (mode == 0) k_zpass<0, E, FZ, 16><<<g, kTpbZ, smem, st>>>(P);
    else k_zpass<1, E, FZ, 16><<<g, kTpbZ, smem, st>>>(P);
  }
}

template <int E, int FZ>
void attrs_zpass(int cap) {
  set_smem_cap(k_zpass<0, E, FZ, 32>, cap);
  set_smem_cap(k_zpass<1, E, FZ, 32>, cap);
  set_smem_cap(k_zpass<0, E, FZ, 16>, cap);
  set_smem_cap(k_zpass<1, E, FZ, 16>, cap);
}

template void launch_zpass<FWI_E, FWI_N>(int, int, dim3, size_t, cudaStream_t, const StepParams&);
template void attrs_zpass<FWI_E, FWI_N>(int);

}  // namespace fwi
