// kp_gmres.cu -- batched restarted GMRES(m) for the five-point Fokker-Planck
// systems of Sec. 2.3 (Eq. 11-13), FP64, one thread block per system: the
// lean instantiations of the kernel in kp_gmres_kernel.cuh, the operator /
// right-hand-side kernel, and the launch helpers of the march.
#include "kp_gmres_kernel.cuh"

namespace kp {
namespace {

// y = A x (mode 0) or b = m^{n-1}/dt - Div_h f (mode 1), one block per system.
__global__ void apply_rhs_kernel(const SysDesc* sys, int nsys, int mode) {
  const SysDesc d = sys[blockIdx.x];
  const int H = d.H, W = d.W, N = H * W;
  const double hh = d.h;
  const double cc = d.g2 / (2.0 * hh * hh);
  const double ee = d.g2 / (8.0 * hh * hh);
  const double cd = 1.0 / d.dt + 2.0 * d.g2 / (hh * hh);
  const double i2h = 1.0 / (2.0 * hh);
  for (int pp = threadIdx.x; pp < N; pp += blockDim.x) {
    const int i = pp / H, j = pp - i * H;
    if (mode == 2) {                      // x <- b - x
      d.x[pp] = d.b[pp] - d.x[pp];
      continue;
    }
    if (mode == 1) {
      const double fE = (d.fx && i + 1 < W) ? d.fx[pp + H] : 0.0;
      const double fW = (d.fx && i > 0) ? d.fx[pp - H] : 0.0;
      const double fN = (d.fy && j + 1 < H) ? d.fy[pp + 1] : 0.0;
      const double fS = (d.fy && j > 0) ? d.fy[pp - 1] : 0.0;
      d.x[pp] = d.b[pp] / d.dt - ((fE - fW) + (fN - fS)) * i2h;
      continue;
    }
    const double mE = (i + 1 < W) ? d.mt[pp + H] : 0.0;
    const double mW = (i > 0) ? d.mt[pp - H] : 0.0;
    const double mN = (j + 1 < H) ? d.mt[pp + 1] : 0.0;
    const double mS = (j > 0) ? d.mt[pp - 1] : 0.0;
    const double fxp = d.fx ? d.fx[pp] : 0.0;
    const double fyp = d.fy ? d.fy[pp] : 0.0;
    const double dmx = mE - mW, dmy = mN - mS;
    double y = cd * d.b[pp];
    if (i + 1 < W) y += (-cc + fxp * i2h - ee * dmx) * d.b[pp + H];
    if (i > 0) y += (-cc - fxp * i2h + ee * dmx) * d.b[pp - H];
    if (j + 1 < H) y += (-cc + fyp * i2h - ee * dmy) * d.b[pp + 1];
    if (j > 0) y += (-cc - fyp * i2h + ee * dmy) * d.b[pp - 1];
    d.x[pp] = y;
  }
}

}  // namespace

size_t gmres_fp64_smem_bytes(int ept, int nt, int S, int m) {
  const int npad = ept * nt;
  const size_t doubles = (size_t)S * npad + npad + (nt / 32) * kMaxV + kMaxV +
                         (size_t)(m + 1) * m + (m + 1) + 4 * m + 8;
  return doubles * sizeof(double) + 8 * sizeof(int);
}

cudaError_t launch_gmres_fp64(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                              cudaStream_t st) {
  if (p.bicg && p.capV) return launch_gmres_fp64_bicg(p, ept, nt, minb, smem, st);
  const int nfeat = (p.score_stride != 0) + (p.dense_slots != 0) + (p.picard > 1);
  if (p.x0_mode == X0_GALERKIN || nfeat > 1) return launch_gmres_fp64_feat(p, ept, nt, minb, smem, st);
  if (p.picard > 1) return launch_gmres_fp64_picard(p, ept, nt, minb, smem, st);
  if (p.score_stride) return launch_gmres_fp64_score(p, ept, nt, minb, smem, st);
  if (p.dense_slots) return launch_gmres_fp64_dense(p, ept, nt, minb, smem, st);
  if (ept == 4 && nt == 256 && minb == 2) return launch_one<4, 256, 2, kVarLean>(p, smem, st);
  if (ept == 4 && nt == 256 && minb == 3) return launch_one<4, 256, 3, kVarLean>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 2) return launch_one<8, 128, 2, kVarLean>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 3) return launch_one<8, 128, 3, kVarLean>(p, smem, st);
  if (ept == 8 && nt == 128 && minb == 4) return launch_one<8, 128, 4, kVarLean>(p, smem, st);
  if (ept == 16 && nt == 64 && minb == 4) return launch_one<16, 64, 4, kVarLean>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1, kVarLean>(p, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_gmres_fp64_1k_grid(const GmresParams& p, size_t smem, int grid,
                                      cudaStream_t st) {
  auto k = gmres_fp64_kernel<4, 256, 2, kVarLean>;
  cudaError_t e = allow_max_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, smem, st>>>(p);
  return cudaGetLastError();
}

__global__ void advance_kernel(int* step, int by, int* zero, int nzero) {
  *step += by;
  for (int k = 0; zero && k < nzero; ++k) zero[k] = 0;
}

cudaError_t launch_advance(int* step, cudaStream_t st, int by, int* zero, int nzero) {
  advance_kernel<<<1, 1, 0, st>>>(step, by, zero, nzero);
  return cudaGetLastError();
}

int gmres_fp64_blocks_per_sm(int ept, int nt, int minb, size_t smem) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  auto occ = [&](auto k, int threads) {
    e = allow_max_smem(k, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem);
  };
  if (ept == 4 && nt == 256 && minb == 2) occ(gmres_fp64_kernel<4, 256, 2, kVarLean>, 256);
  else if (ept == 4 && nt == 256 && minb == 3) occ(gmres_fp64_kernel<4, 256, 3, kVarLean>, 256);
  else if (ept == 8 && nt == 128 && minb == 2) occ(gmres_fp64_kernel<8, 128, 2, kVarLean>, 128);
  else if (ept == 8 && nt == 128 && minb == 3) occ(gmres_fp64_kernel<8, 128, 3, kVarLean>, 128);
  else if (ept == 8 && nt == 128 && minb == 4) occ(gmres_fp64_kernel<8, 128, 4, kVarLean>, 128);
  else if (ept == 16 && nt == 64 && minb == 4) occ(gmres_fp64_kernel<16, 64, 4, kVarLean>, 64);
  else if (ept == 8 && nt == 512) occ(gmres_fp64_kernel<8, 512, 1, kVarLean>, 512);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_apply(const SysDesc* sys, int nsys, int mode, cudaStream_t st) {
  apply_rhs_kernel<<<nsys, 256, 0, st>>>(sys, nsys, mode);
  return cudaGetLastError();
}

}  // namespace kp
