// kp_internal.cuh -- device-side types and helpers shared by the solver kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kp.h"

namespace kp {

// Per-system descriptor as the kernels read it (built by the host from kp_op
// and the caller's pointer arrays).  `b` is the right-hand side (solvers), the
// vector to project (projection) or m^{n-1} (rhs kernel); `x` is in/out.
struct SysDesc {
  const double* mt;
  const double* fx;
  const double* fy;
  const double* b;
  double* x;
  int H, W;
  double dt, g2, h;
  int slot;   // basis slot (projection) / unused
  int pad_;
};

// Metadata of one stored seed basis.
struct SlotMeta {
  int a;          // basis vectors used (a')
  int has_next;   // v_{a'+1} kept
  int timestep;   // timestep the basis belongs to (-1 = empty)
  int N;
  int lsq;        // projection solves the (a'+1) x a' least-squares problem
  int nrot;       // Givens rotations applied to c before the triangular solve
  int pad_[2];
};

// Capture record of one seed system after kp_seed_solve.
struct CapMeta {
  int a;
  int has_next;
  int N;
  int valid;
};

constexpr int kMaxM = 64;            // largest restart length / basis size
constexpr int kMaxV = kMaxM + 8;     // values per block reduction

struct GmresParams {
  const SysDesc* sys;
  int nsys;
  double tol;
  int m;
  int maxit;
  int S;            // Krylov vectors held in shared memory
  int reorth;       // 0 CGS2, 1 DGKS-conditional second pass
  int npad;         // padded vector length (EPT * NT)
  double* spill;    // [gridDim.x][m + 1 - S][npad] device workspace, or null
  kp_info* info;    // [nsys] or null
  // first-cycle capture (seed solve); capV null = no capture
  double* capV;     // [nsys][cap_a + 1][cap_ld]
  double* capH;     // [nsys][(cap_a + 1) * cap_a] column-major, ld cap_a + 1
  CapMeta* capMeta; // [nsys]
  int cap_a;
  int cap_ld;
  // time march: timestep index and g^2 schedule in device memory (graph replay)
  const int* step;          // null = not marching
  const double* g2_sched;   // if step: g2 = g2_sched[*step] for every system
};

struct ProjParams {
  const SysDesc* sys;
  int nt;
  int timestep;
  const double* slotV;     // [max_seeds][max_a + 1][ld]
  const SlotMeta* meta;    // [max_seeds]
  const double* slotR;     // [max_seeds][(max_a + 1) * max_a] col-major R factor, ld max_a + 1
  const double* slotRot;   // [max_seeds][2 * max_a] (c, s) pairs
  int max_a;
  int ld;
  const int* step;         // if non-null, the timestep is *step
};

struct FactorParams {
  const double* capV;
  const double* capH;
  const CapMeta* capMeta;
  int sys;
  int cap_a;
  int cap_ld;
  double* slotV;
  SlotMeta* meta;
  double* slotR;
  double* slotRot;
  double* slotH;           // [max_seeds][(max_a + 1) * max_a] unrotated Hbar copy
  int seed_id;             // block b stores capture sys + b into slot seed_id + b
  int timestep;
  int max_a;
  int ld;
  int count;               // number of (sys, slot) pairs, one block each
  const int* step;         // if non-null, the timestep is *step
};

// ---- block reductions shared by the kernels ----

constexpr unsigned kFull = 0xffffffffu;

// Warp reduce-scatter of 8 values per lane.  Lanes with (lane & 3) == 0 end
// with the warp sum of value index 4*bit4 + 2*bit3 + bit2 of their lane id.
__device__ __forceinline__ double warp_reduce8(double (&a)[8], int lane) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 16;
    const double send = up ? a[k] : a[k + 4];
    const double keep = up ? a[k + 4] : a[k];
    a[k] = keep + __shfl_xor_sync(kFull, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 8;
    const double send = up ? a[k] : a[k + 2];
    const double keep = up ? a[k + 2] : a[k];
    a[k] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  {
    const bool up = lane & 4;
    const double send = up ? a[0] : a[1];
    const double keep = up ? a[1] : a[0];
    a[0] = keep + __shfl_xor_sync(kFull, send, 4);
  }
  a[0] += __shfl_xor_sync(kFull, a[0], 2);
  a[0] += __shfl_xor_sync(kFull, a[0], 1);
  return a[0];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Per-warp partial sums of nv values partial(i) into red[warp][i]; ends with
// a block barrier.  Every thread must call it with the same nv.
template <int NT, typename F>
__device__ __forceinline__ void block_partials(int nv, F&& partial, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (i0 + k < nv) ? partial(i0 + k) : 0.0;
    const double s = warp_reduce8(a, lane);
    const int v = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && i0 + v < nv) red[warp * kMaxV + i0 + v] = s;
  }
  __syncthreads();
}

// Cross-warp sum of value i (called by warp 0 lanes).
template <int NT>
__device__ __forceinline__ double cross_warp(const double* red, int i) {
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w * kMaxV + i];
  return s;
}

// Launchers (defined in the .cu files; return a cudaError_t of the launch).
cudaError_t launch_gmres_fp64(const GmresParams& p, int ept, int nt, size_t smem,
                              cudaStream_t st);
size_t gmres_fp64_smem_bytes(int ept, int nt, int S, int m);
// The N <= 1024 instantiation (4 points x 256 threads) on an explicit grid;
// the kernel strides over systems, block b using Krylov workspace slice b.
cudaError_t launch_gmres_fp64_1k_grid(const GmresParams& p, size_t smem, int grid,
                                      cudaStream_t st);
cudaError_t launch_apply(const SysDesc* sys, int nsys, int mode, cudaStream_t st);
cudaError_t launch_factor(const FactorParams& p, cudaStream_t st);
cudaError_t launch_project_fp64(const ProjParams& p, int ept, int nt, cudaStream_t st);

}  // namespace kp
