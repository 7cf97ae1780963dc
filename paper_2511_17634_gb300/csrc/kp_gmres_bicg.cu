// kp_gmres_bicg.cu -- the kVarBicg instantiations of the FP64 solver kernel
// (kp_gmres_kernel.cuh): seed solves by BiCGSTAB (Sec. 3, Phase 1 as the paper
// states it) with the key-vector basis and the explicit A_proj, used by the
// seed launches of a march that asks for them.
#include "kp_gmres_kernel.cuh"

namespace kp {

cudaError_t launch_gmres_fp64_bicg(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st) {
  if (ept == 4 && nt == 256 && minb == 2) return launch_one<4, 256, 2, kVarBicg>(p, smem, st);
  if (ept == 4 && nt == 256 && minb == 3) return launch_one<4, 256, 3, kVarBicg>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 2) return launch_one<8, 128, 2, kVarBicg>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 3) return launch_one<8, 128, 3, kVarBicg>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 4) return launch_one<8, 128, 4, kVarBicg>(p, smem, st);
  if (ept == 16 && nt == 64 && minb == 4) return launch_one<16, 64, 4, kVarBicg>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1, kVarBicg>(p, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
