// kp_gmres_picard.cu -- the kVarPicard instantiations of the FP64 solver kernel
// (kp_gmres_kernel.cuh): the plain solver plus K > 1 Picard iterations of the
// lagged linearisation per timestep (Sec. 2.3), used by the launches of
// marches that ask for them.
#include "kp_gmres_kernel.cuh"

namespace kp {

cudaError_t launch_gmres_fp64_picard(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st) {
  if (ept == 4 && nt == 256 && minb == 2) return launch_one<4, 256, 2, kVarPicard>(p, smem, st);
  if (ept == 4 && nt == 256 && minb == 3) return launch_one<4, 256, 3, kVarPicard>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 2) return launch_one<8, 128, 2, kVarPicard>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 3) return launch_one<8, 128, 3, kVarPicard>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 4) return launch_one<8, 128, 4, kVarPicard>(p, smem, st);
  if (ept == 16 && nt == 64 && minb == 4) return launch_one<16, 64, 4, kVarPicard>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1, kVarPicard>(p, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
