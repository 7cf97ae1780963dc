// kp_ctx.h -- host-side context shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "kp.h"
#include "kp_internal.cuh"

namespace kp {

constexpr int kRing = 8;

struct Staging {
  SysDesc* host = nullptr;   // pinned
  size_t cap = 0;
  cudaEvent_t done = nullptr;
  bool pending = false;
};

}  // namespace kp

struct kp_ctx {
  kp_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  size_t smem_optin = 0;
  char err[512] = {0};

  // per-call descriptor upload: pinned host ring -> device buffer
  kp::Staging ring[kp::kRing];
  int ring_next = 0;
  kp::SysDesc* d_desc = nullptr;
  size_t d_desc_cap = 0;

  // first-cycle capture of the last seed solve
  double* capV = nullptr;
  double* capH = nullptr;
  kp::CapMeta* capMeta = nullptr;
  int cap_nsys = 0;       // capacity in systems
  int cap_last = 0;       // systems in the last seed solve

  // seed-basis store
  double* slotV = nullptr;
  float* slotV32 = nullptr;   // mixed precision: FP32 seed bases
  __nv_bfloat16* slotVb = nullptr;   // mixed precision: BF16 seed bases [slot][48][vb_ld]
  int vb_ld = 0;
  float* capV32 = nullptr;    // mixed precision: FP32 capture
  kp::SlotMeta* slotMeta = nullptr;
  double* slotR = nullptr;
  double* slotRot = nullptr;
  double* slotH = nullptr;
  std::vector<int> slot_timestep;
  std::vector<int> slot_n;

  // Krylov-vector workspace for vectors that do not fit in shared memory
  double* spill = nullptr;
  kp::ProjTile* d_tiles = nullptr;   // tile list of the projection GEMM
  size_t d_tiles_bytes = 0;
  int* d_err = nullptr;               // device error flag of bounded waits
  float* spill32 = nullptr;
  size_t spill32_bytes = 0;
  size_t spill_bytes = 0;
};


namespace kp {

// Launch shape of the GMRES kernel family for systems of up to nmax unknowns.
struct Shape {
  int ept = 0, nt = 0, S = 0;
  int minb = 1;   // resident blocks per SM the kernel is compiled for (launch bounds)
  size_t smem = 0;
  int cs = 0;   // > 0: thread-block cluster of cs CTAs per system (slices of W/cs columns)
};

kp_status set_error(kp_ctx* c, kp_status s, const char* fmt, ...);
kp_status cuda_error(kp_ctx* c, cudaError_t e, const char* what);
// Chooses threads, elements per thread and the shared-memory Krylov window
// (FP64 vectors, or FP32 ones for the mixed-precision solver).
kp_status gmres_shape(kp_ctx* c, int nmax, int m, Shape* out, bool mixed = false,
                      int wmin = 0);
// Inner FP32 residual reduction of the mixed-precision solvers.
inline double inner_eta(const kp_options& o) {
  static const double k[8] = {1e-5, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7};
  return k[o.inner_digits >= 0 && o.inner_digits <= 7 ? o.inner_digits : 0];
}

// Launch the solver kernel family that `sh` selects.
cudaError_t launch_solver(const GmresParams& p, const Shape& sh, bool mixed, cudaStream_t st);

// Learned initial guess inside the time march (kp_cnn.cu): whether the
// network can serve an H x W march (10 inputs, 1 output, implicit-GEMM
// inference buffers), how many images one pass holds, and the enqueue of
// the network's part of x[b] = mprev[b] + dt rho_b net(mprev[b], mseed[b],
// time planes, r_hat) for B targets (device pointer tables; timestep from the
// device counter): net -> delta[b * H W ..] (FP32) and rho_b -> rho[b]; the
// solver forms x from them.
bool cnn_march_ready(const kp_cnn* n, int H, int W);
int cnn_inference_batch(const kp_cnn* n);
cudaError_t cnn_enqueue_guess(kp_cnn* n, int B, const double* const* mprev, const double* const* mseed,
                              float* delta, double* rho, const int* step, int step_offset, const double* g2,
                              int T, cudaStream_t st);

}  // namespace kp
