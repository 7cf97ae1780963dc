// kp_gmres_dense.cu -- the kVarDense instantiations of the FP64 solver kernel
// (kp_gmres_kernel.cuh): the plain solver plus the projection through an
// explicit A_proj (Sec. 3, Phase 2), used by the target launches of marches
// whose seed bases are BiCGSTAB key vectors or cycled (accumulated) bases.
#include "kp_gmres_kernel.cuh"

namespace kp {

cudaError_t launch_gmres_fp64_dense(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st) {
  if (ept == 4 && nt == 256 && minb == 2) return launch_one<4, 256, 2, kVarDense>(p, smem, st);
  if (ept == 4 && nt == 256 && minb == 3) return launch_one<4, 256, 3, kVarDense>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 2) return launch_one<8, 128, 2, kVarDense>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 3) return launch_one<8, 128, 3, kVarDense>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 4) return launch_one<8, 128, 4, kVarDense>(p, smem, st);
  if (ept == 16 && nt == 64 && minb == 4) return launch_one<16, 64, 4, kVarDense>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1, kVarDense>(p, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
