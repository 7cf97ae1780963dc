// kp_gmres_feat.cu -- the FEAT instantiations of the FP64 GMRES kernel
// (kp_gmres_kernel.cuh): exact-Galerkin initial guess, Picard iterations and
// the fused score / embedding epilogue, used only when a launch asks for one.
#include "kp_gmres_kernel.cuh"

namespace kp {

cudaError_t launch_gmres_fp64_feat(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st) {
  if (ept == 4 && nt == 256 && minb == 2) return launch_one<4, 256, 2, true>(p, smem, st);
  if (ept == 4 && nt == 256 && minb == 3) return launch_one<4, 256, 3, true>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 2) return launch_one<8, 128, 2, true>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 3) return launch_one<8, 128, 3, true>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 4) return launch_one<8, 128, 4, true>(p, smem, st);
  if (ept == 16 && nt == 64 && minb == 4) return launch_one<16, 64, 4, true>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1, true>(p, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
