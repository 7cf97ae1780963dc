// kp_gmres_feat.cu -- the kVarFeat instantiations of the FP64 GMRES kernel
// (kp_gmres_kernel.cuh): exact-Galerkin initial guess, Picard iterations, the
// fused score / embedding epilogue and the projection through an explicit
// A_proj (BiCGSTAB seed bases), used only when a launch asks for one.
#include "kp_gmres_kernel.cuh"

namespace kp {

cudaError_t launch_gmres_fp64_feat(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st) {
  if (ept == 4 && nt == 256 && minb == 2) return launch_one<4, 256, 2, kVarFeat>(p, smem, st);
  if (ept == 4 && nt == 256 && minb == 3) return launch_one<4, 256, 3, kVarFeat>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 2) return launch_one<8, 128, 2, kVarFeat>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 3) return launch_one<8, 128, 3, kVarFeat>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 4) return launch_one<8, 128, 4, kVarFeat>(p, smem, st);
  if (ept == 16 && nt == 64 && minb == 4) return launch_one<16, 64, 4, kVarFeat>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1, kVarFeat>(p, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
