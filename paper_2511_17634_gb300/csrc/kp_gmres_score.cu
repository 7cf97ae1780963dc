// kp_gmres_score.cu -- the kVarScore instantiations of the FP64 solver kernel
// (kp_gmres_kernel.cuh): the plain solver plus the fused epilogue that writes
// the score of every solved timestep and advances the probability-flow
// embedding (end of Sec. 2.3, Sec. 4.1), used by the target launches of
// marches that keep the score.
#include "kp_gmres_kernel.cuh"

namespace kp {

cudaError_t launch_gmres_fp64_score(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st) {
  if (ept == 4 && nt == 256 && minb == 2) return launch_one<4, 256, 2, kVarScore>(p, smem, st);
  if (ept == 4 && nt == 256 && minb == 3) return launch_one<4, 256, 3, kVarScore>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 2) return launch_one<8, 128, 2, kVarScore>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 3) return launch_one<8, 128, 3, kVarScore>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 4) return launch_one<8, 128, 4, kVarScore>(p, smem, st);
  if (ept == 16 && nt == 64 && minb == 4) return launch_one<16, 64, 4, kVarScore>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1, kVarScore>(p, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
