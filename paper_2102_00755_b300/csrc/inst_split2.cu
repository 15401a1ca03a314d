// Instantiations of the two-step split-plane kernels for one square plane side, FWI_N.
#include "launch.cuh"
#include "split2.cuh"

namespace fwi {

template <int N>
void launch_split2(int kind, dim3 g, size_t smem, cudaStream_t st, const StepParams& P) {
  constexpr int TY = ty2_for(N), NPC = npc2_for(N);
  constexpr int NTY = Y2<N, TY>::NT, NTX = X2<N, NPC>::NT;
  switch (kind) {
    case 0: k_ypass2<Y_INV_MOM, N, TY><<<g, NTY, smem, st>>>(P); break;
    case 1: k_ypass2<Y_INV_MASS, N, TY><<<g, NTY, smem, st>>>(P); break;
    case 2: k_ypass2<Y_FWD3, N, TY><<<g, NTY, smem, st>>>(P); break;
    case 3: k_ypass2<Y_FWD1, N, TY><<<g, NTY, smem, st>>>(P); break;
    case 4: k_xpass2_mom<N, NPC><<<g, NTX, smem, st>>>(P); break;
    default: k_xpass2_mass<N, NPC><<<g, NTX, smem, st>>>(P); break;
  }
}

template <int N>
void attrs_split2(int cap) {
  constexpr int TY = ty2_for(N), NPC = npc2_for(N);
  set_smem_cap(k_ypass2<Y_INV_MOM, N, TY>, cap);
  set_smem_cap(k_ypass2<Y_INV_MASS, N, TY>, cap);
  set_smem_cap(k_ypass2<Y_FWD3, N, TY>, cap);
  set_smem_cap(k_ypass2<Y_FWD1, N, TY>, cap);
  set_smem_cap(k_xpass2_mom<N, NPC>, cap);
  set_smem_cap(k_xpass2_mass<N, NPC>, cap);
}

template void launch_split2<FWI_N>(int, dim3, size_t, cudaStream_t, const StepParams&);
template void attrs_split2<FWI_N>(int);

}  // namespace fwi
