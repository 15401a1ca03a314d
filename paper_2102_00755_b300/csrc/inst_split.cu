// Instantiations of the warp-owned split-plane kernels with FWI_E values staged per lane.
#include "launch.cuh"

namespace fwi {

template <int E>
void launch_split(int kind, dim3 g, size_t smem, cudaStream_t st, const StepParams& P) {
  switch (kind) {
    case 0: k_ypass<Y_INV_MOM, E><<<g, kTpbZ, smem, st>>>(P); break;
    case 1: k_ypass<Y_INV_MASS, E><<<g, kTpbZ, smem, st>>>(P); break;
    case 2: k_ypass<Y_FWD3, E><<<g, kTpbZ, smem, st>>>(P); break;
    case 3: k_ypass<Y_FWD1, E><<<g, kTpbZ, smem, st>>>(P); break;
    case 4: k_xpass_mom<E><<<g, kTpbPlane, smem, st>>>(P); break;
    case 5: k_xpass_mass<E><<<g, kTpbPlane, smem, st>>>(P); break;
    default: k_xpass_tr_init<E><<<g, kTpbPlane, smem, st>>>(P); break;
  }
}

template <int E>
void attrs_split(int cap) {
  set_smem_cap(k_ypass<Y_INV_MOM, E>, cap);
  set_smem_cap(k_ypass<Y_INV_MASS, E>, cap);
  set_smem_cap(k_ypass<Y_FWD3, E>, cap);
  set_smem_cap(k_ypass<Y_FWD1, E>, cap);
  set_smem_cap(k_xpass_mom<E>, cap);
  set_smem_cap(k_xpass_mass<E>, cap);
  set_smem_cap(k_xpass_tr_init<E>, cap);
}

template void launch_split<FWI_E>(int, dim3, size_t, cudaStream_t, const StepParams&);
template void attrs_split<FWI_E>(int);

}  // namespace fwi
