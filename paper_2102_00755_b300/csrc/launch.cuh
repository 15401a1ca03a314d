// Launchers of the step kernels.  Each kernel family's instantiations live in a
// translation unit of their own (inst_*.cu, compiled once per size with -DFWI_N /
// -DFWI_E), so that the library compiles in parallel; fwi.cu sees only these
// declarations.  Every launcher picks its kernel's block size itself and takes
// the grid, the dynamic shared memory and the stream from the caller.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fwi {

// Raise a kernel's dynamic shared-memory limit to the device's per-block opt-in maximum
// `cap` less the kernel's static shared memory (static + dynamic may not exceed cap).
template <class F>
void set_smem_cap(F* f, int cap) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, f) == cudaSuccess) cap -= (int)a.sharedSizeBytes;
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

// two-step plane kernels for square planes of side N (plane2.cuh):
// kind 0 = k_plane2_mom, 1 = k_plane2_mass
template <int N> void launch_plane2(int kind, dim3 grid, size_t smem, cudaStream_t st, const StepParams& P);
template <int N> void attrs_plane2(int cap);

// two-step z pass for nz = NZ (plane2.cuh): mode 0 = momentum, 1 = mass; tz = 16 or 32
template <int NZ> void launch_zpass2(int mode, int tz, dim3 grid, size_t smem, cudaStream_t st,
                                     const StepParams& P);
template <int NZ> void attrs_zpass2(int cap);

// two-step split planes of side N (split2.cuh): kind 0..3 = k_ypass2 of YKind 0..3,
// 4 = k_xpass2_mom, 5 = k_xpass2_mass
template <int N> void launch_split2(int kind, dim3 grid, size_t smem, cudaStream_t st, const StepParams& P);
template <int N> void attrs_split2(int cap);

// warp-owned z pass (kernels.cuh): FZ = compile-time length or 0 (runtime radix
// schedule, E values staged per lane); mode 0 = momentum, 1 = mass; tz = 16 or 32
template <int E, int FZ> void launch_zpass(int mode, int tz, dim3 grid, size_t smem, cudaStream_t st,
                                           const StepParams& P);
template <int E, int FZ> void attrs_zpass(int cap);

// warp-owned plane kernels (kernels.cuh): kind 0 = k_plane_mom, 1 = k_plane_mass, 2 = k_tr_init
template <int E, int F> void launch_plane(int kind, dim3 grid, size_t smem, cudaStream_t st, const StepParams& P);
template <int E, int F> void attrs_plane(int cap);

// warp-owned split planes (kernels.cuh): kind 0..3 = k_ypass of YKind 0..3,
// 4 = k_xpass_mom, 5 = k_xpass_mass, 6 = k_xpass_tr_init
template <int E> void launch_split(int kind, dim3 grid, size_t smem, cudaStream_t st, const StepParams& P);
template <int E> void attrs_split(int cap);

}  // namespace fwi
