// kp_internal.cuh -- device-side types and helpers shared by the solver kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
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
  double* score;   // march targets, optional: this system's [2][N] score plane set of timestep 0
  double* emb;     // march targets, optional: this system's [2][N] probability-flow embedding
};

// Metadata of one stored seed basis.
struct SlotMeta {
  int a;          // basis vectors used (a')
  int has_next;   // v_{a'+1} kept
  int timestep;   // timestep the basis belongs to (-1 = empty)
  int N;
  int lsq;        // projection solves the (a'+1) x a' least-squares problem
  int nrot;       // Givens rotations applied to c before the triangular solve
  int dense;      // 1: slotR holds the explicit A_proj = V^T A_seed V (a x a,
                  // ld max_a + 1) of a BiCGSTAB basis instead of a QR of H_a
  int pad_;
};

// Per-timestep totals accumulated by the solver blocks (time march).
struct StepAcc {
  unsigned long long seed_iters;
  unsigned long long tgt_iters;
  unsigned long long seed_flops;     // FP64 flops of the algorithm (see gmres_flops)
  unsigned long long tgt_flops;
  unsigned long long proj_flops;
  unsigned long long tgt_flops32;    // FP32 Krylov flops of mixed-precision target solves
  unsigned long long max_res_bits;   // max relative residual (non-negative double bits)
  unsigned int tgt_max_iters;
  unsigned int not_converged;
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
// Mixed precision: an inner FP32 GMRES cycle stops once its residual estimate
// is below max(eta beta, kInnerFloor tol ||b||).  The estimate tracks the true
// residual to about 1e-7 of the cycle's starting residual (FP32 rounding of
// the correction), so a floor at half the outer tolerance lets the true
// residual that follows meet tol without solving the last cycle further down.
constexpr double kInnerFloor = 0.5;

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
  double* capM;     // seed cycling: [slot][cap_ld] the lagged field m~ of the
                    // solve that filled the slot (its operator), or null
  CapMeta* capMeta; // [nsys]
  int cap_a;
  int cap_ld;
  int fixed_a;      // 1: the capture cycle takes min(cap_a, m) steps before the
                    // residual test may end it (fixed basis dimension, Sec. 3)
  double inner_eta; // mixed precision: inner FP32 residual reduction per outer step (0 = 1e-5)
  // time march: timestep index and g^2 schedule in device memory (graph replay)
  const int* step;          // null = not marching
  const double* g2_sched;   // if step: g2 = g2_sched[*step + step_offset] for every system
  int step_offset;          // seeds run one timestep ahead of the targets
  const int* step_end;      // if step: nothing to do when *step + step_offset >= *step_end
  double b_scale;           // right-hand side = b[p] * b_scale (b = m^{n-1}/dt when f = 0)
  int x0_mode;              // X0_* below
  // seed-basis store: projection source (X0_PROJECT) and fused capture (factor)
  double* slotV;            // [max_seeds][max_a + 1][slot_ld]
  SlotMeta* slotMeta;
  double* slotR;
  double* slotRot;
  int slot_ld;
  int max_a;
  int slot_parity_stride;   // slots of timestep parity q start at q * stride
  int factor;               // capture into slot (sys + parity offset) and factor H_a
  StepAcc* acc;             // per-timestep totals (indexed like g2_sched) or null
  int acc_kind;             // 0 seeds, 1 targets
  // mixed precision (FP32 Krylov vectors)
  float* spill32;           // [gridDim.x][m + 1 - S][npad] workspace
  float* capV32;            // capture target for FP32 bases (slot layout when factor)
  const float* slotV32;     // [max_seeds][max_a + 1][slot_ld] FP32 seed bases
  const float* cproj;       // if set: c = V^T b per target, [nsys][cproj_ld] (tensor-core GEMM)
  int cproj_ld;
  __nv_bfloat16* bnext;     // if set: write BF16 (x * b_scale) per system, [nsys][bnext_ld]
  int bnext_ld;
  __nv_bfloat16* capVb;     // if set: BF16 copy of the captured basis, [slot][kVbRows][capVb_ld]
  int capVb_ld;
  // march windows (FP64 solver): one launch covers timesteps
  // *step + step_offset .. + win - 1 (clipped at *step_end)
  int win;                  // 0 = one timestep per launch
  int slot_sets;            // seed-slot sets: timestep t uses set t % slot_sets (0 = 2)
  const SysDesc* sys_par[2];// if set: timestep t uses sys_par[(t + sys_shift) & 1] (else sys)
  int sys_shift;
  int* queue;               // dynamic schedule: item counter (zeroed before the launch);
                            // null = static (each block marches its systems through the window)
  int* done;                // [nsys] timesteps completed since *run_start (dynamic schedule)
  const int* run_start;
  int wait_bias;            // testing aid: added to every awaited count (1: never released)
  int wait_limit;           // polls before a wait gives up; 0 = kWaitLimit
  int* err;                 // bit 1: a dependency wait gave up
  int grid;                 // blocks of the launch (0 = one per system)
  size_t score_stride;      // > 0: write the score of each solved timestep to
                            // d.score + tstep * score_stride and advance d.emb
  int picard;               // > 1: Picard iterations per system (FP64 solver)
  int bicg;                 // 1: seed solves by BiCGSTAB (dense A_proj slots)
  int dense_slots;          // targets: slots may hold an explicit A_proj (BiCGSTAB
                            // seeds, seed cycling): the feature variant projects
  int pdl;                  // programmatic launch, bit 0: let the stream's next launch
                            // start at once; bit 1: launched that way, wait for the
                            // prior grid (its completion and memory) before exiting
  // exact Galerkin in mixed precision (X0_GALERKIN, one-block mixed solver):
  // G_i[p][q] = gram0[slot][p * gram_a + q] + gram[target][p * gram_a + q]
  // (kp_gram.cu), c = V^T b in cproj
  const float* gram0;
  const float* gram;
  int gram_a;
  // learned guess (X0_READ / X0_GUESS_PROJECT in a march): if gdelta is set,
  // x_init of system s is m~ + (grho[s] / gdiv) gdelta[s * gdelta_ld + p]
  // (the network's output in units of dt rho, gdiv = T), formed in the solver
  const float* gdelta;
  int gdelta_ld;
  const double* grho;
  double gdiv;
};

constexpr int kWaitLimit = 1 << 22;   // polls (>= 256 ns apart) before a wait gives up

// First seed slot of timestep t (slot sets rotate with the timestep).
__host__ __device__ inline int slot_set_base(const GmresParams& p, int t) {
  const int sets = p.slot_sets > 2 ? p.slot_sets : 2;
  return (t % sets) * p.slot_parity_stride;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* a) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int* a, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

constexpr int kVbRows = 48;   // rows per seed slot of the BF16 basis (tensor-core N tile)

// X0_GUESS_PROJECT: x_init is read from x; x0 = x_init + V_a H_a^{-1} V_a^T
// (b - A x_init), the projection of Sec. 3 applied to the guess's residual
// (mixed-precision solvers)
enum { X0_READ = 0, X0_ZERO = 1, X0_WARM = 2, X0_PROJECT = 3, X0_GALERKIN = 4, X0_GUESS_PROJECT = 5 };

// Solves G y = c (G: n x n column-major in shared memory, c: length n) by LU
// with partial pivoting on one warp (lanes own rows); y overwrites c, G is
// overwritten.  Returns false (on every lane) if a pivot is exactly zero.
__device__ __forceinline__ bool lu_solve_warp(double* G, int n, double* c, int lane) {
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + lane; i < n; i += 32) {
      const double v = fabs(G[i + k * n]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (!(best > 0.0)) return false;
    if (bi != k) {
      for (int j = lane; j < n; j += 32) {
        const double t = G[k + j * n];
        G[k + j * n] = G[bi + j * n];
        G[bi + j * n] = t;
      }
      if (lane == 0) { const double t = c[k]; c[k] = c[bi]; c[bi] = t; }
    }
    __syncwarp();
    const double ip = 1.0 / G[k + k * n];
    for (int i = k + 1 + lane; i < n; i += 32) {
      const double l = G[i + k * n] * ip;
      for (int j = k + 1; j < n; ++j) G[i + j * n] = fma(-l, G[k + j * n], G[i + j * n]);
      c[i] = fma(-l, c[k], c[i]);
    }
    __syncwarp();
  }
  if (lane == 0)
    for (int i = n - 1; i >= 0; --i) {
      double s = c[i];
      for (int j = i + 1; j < n; ++j) s = fma(-G[i + j * n], c[j], s);
      c[i] = s / G[i + i * n];
    }
  __syncwarp();
  return true;
}

struct ProjParams {
  const SysDesc* sys;
  int nt;
  int timestep;
  const double* slotV;     // [max_seeds][max_a + 1][ld]
  const SlotMeta* meta;    // [max_seeds]
  const double* slotR;     // [max_seeds][(max_a + 1) * max_a] col-major R factor, ld max_a + 1
  const double* slotRot;   // [max_seeds][3 * max_a]: (c, s) pairs, then reciprocal pivots
  int max_a;
  int ld;
  const int* step;         // if non-null, the timestep is *step
  const float* slotV32;    // mixed precision: FP32 bases instead of slotV
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
  const float* capV32;     // mixed precision: FP32 capture and slot bases (else null)
  float* slotV32;
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

// Warp reduce-scatter of 4 values per lane: lanes with (lane & 7) == 0 end
// with the warp sum of value 2*bit4 + bit3 (6 adds instead of 4 x 5).
__device__ __forceinline__ double warp_reduce4(double (&a)[8], int lane) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 16;
    const double send = up ? a[k] : a[k + 2];
    const double keep = up ? a[k + 2] : a[k];
    a[k] = keep + __shfl_xor_sync(kFull, send, 16);
  }
  {
    const bool up = lane & 8;
    const double send = up ? a[0] : a[1];
    const double keep = up ? a[1] : a[0];
    a[0] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  a[0] += __shfl_xor_sync(kFull, a[0], 4);
  a[0] += __shfl_xor_sync(kFull, a[0], 2);
  a[0] += __shfl_xor_sync(kFull, a[0], 1);
  return a[0];
}

// Per-warp partial sums of nv values partial(i) into red[warp][i]; ends with
// a block barrier.  Every thread must call it with the same nv.  Chunks of 8
// values use an 8-wide reduce-scatter, a last chunk of up to 4 a 4-wide one,
// a single value a plain butterfly.
template <int NT, typename F>
__device__ __forceinline__ void block_partials(int nv, F&& partial, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int i0 = 0;
  for (; i0 + 4 < nv; i0 += 8) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (i0 + k < nv) ? partial(i0 + k) : 0.0;
    const double s = warp_reduce8(a, lane);
    const int v = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && i0 + v < nv) red[warp * kMaxV + i0 + v] = s;
  }
  if (i0 + 1 < nv) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = (i0 + k < nv) ? partial(i0 + k) : 0.0;
    const double s = warp_reduce4(a, lane);
    const int v = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
    if ((lane & 7) == 0 && i0 + v < nv) red[warp * kMaxV + i0 + v] = s;
  } else if (i0 < nv) {
    const double s = warp_sum(partial(i0));
    if (lane == 0) red[warp * kMaxV + i0] = s;
  }
  __syncthreads();
}

// FP32 variants for the mixed-precision solver: FP32 partials and warp
// reduce-scatter, FP64 cross-warp sum (cross_warp) afterwards.
__device__ __forceinline__ float warp_reduce8f(float (&a)[8], int lane) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 16;
    const float send = up ? a[k] : a[k + 4];
    const float keep = up ? a[k + 4] : a[k];
    a[k] = keep + __shfl_xor_sync(kFull, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 8;
    const float send = up ? a[k] : a[k + 2];
    const float keep = up ? a[k + 2] : a[k];
    a[k] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  {
    const bool up = lane & 4;
    const float send = up ? a[0] : a[1];
    const float keep = up ? a[1] : a[0];
    a[0] = keep + __shfl_xor_sync(kFull, send, 4);
  }
  a[0] += __shfl_xor_sync(kFull, a[0], 2);
  a[0] += __shfl_xor_sync(kFull, a[0], 1);
  return a[0];
}

template <int NT, typename F>
__device__ __forceinline__ void block_partials_f32(int nv, F&& partial, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (i0 + k < nv) ? partial(i0 + k) : 0.f;
    const float s = warp_reduce8f(a, lane);
    const int v = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && i0 + v < nv) red[warp * kMaxV + i0 + v] = (double)s;
  }
  __syncthreads();
}

// As block_partials_f32, with the per-warp partials kept in FP32 (red32[warp][i]).
template <int NT, typename F>
__device__ __forceinline__ void block_partials_f32x(int nv, F&& partial, float* red32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (i0 + k < nv) ? partial(i0 + k) : 0.f;
    const float s = warp_reduce8f(a, lane);
    const int v = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && i0 + v < nv) red32[warp * kMaxV + i0 + v] = s;
  }
  __syncthreads();
}

// Cross-warp sums of nv values from FP32 partials, by all 32 lanes of one
// warp: each round holds the NT/32 partials of 32/(NT/32) values in lane
// groups and adds them in an FP32 butterfly; dst[i] = the sum, as a double.
// Runs on the FP32 pipe (one conversion per value) instead of NT/32 - 1
// dependent FP64 adds on a few lanes.
template <int NT>
__device__ __forceinline__ void cross_warp_f32(const float* red32, int nv, double* dst, int lane) {
  constexpr int NW = NT / 32;
  constexpr int PER = 32 / NW;
  for (int i0 = 0; i0 < nv; i0 += PER) {
    const int i = i0 + lane / NW, w = lane % NW;
    float v = (i < nv) ? red32[w * kMaxV + i] : 0.f;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (w == 0 && i < nv) dst[i] = (double)v;
  }
}

// Cross-warp sum of value i (called by warp 0 lanes).
template <int NT>
__device__ __forceinline__ double cross_warp(const double* red, int i) {
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w * kMaxV + i];
  return s;
}

// FP64 flops per unknown of GMRES(m) with CGS2 as implemented here, for k
// Arnoldi steps: 14 to start (residual, two norms); per cycle of L steps
// sum_{j<L} (7 shifted stencil + 8(j+1) Gram-Schmidt + 5 norm/scale)
// + 2L update + 12 residual.
__host__ __device__ __forceinline__ unsigned long long gmres_flops(int k, int m) {
  const unsigned long long full = (unsigned long long)(k / m), rem = (unsigned long long)(k % m);
  const unsigned long long M = (unsigned long long)m;
  unsigned long long f = 14ull + full * (4ull * M * M + 18ull * M + 12ull);
  if (rem) f += 4ull * rem * rem + 18ull * rem + 12ull;
  return f;
}

__device__ __forceinline__ void givens_rot(double a, double b, double& c, double& s) {
  if (b == 0.0) { c = 1.0; s = 0.0; return; }
  const double r = hypot(a, b);
  const double ir = 1.0 / r;
  c = a * ir;
  s = b * ir;
}

// Givens QR of a seed's Hessenberg matrix for the projection of Sec. 3
// (one thread).  Hb: unrotated (a+1) x a, column-major, leading dim ld, also
// the leading dim of R.  First tries H_a (a-1 rotations); if a pivot is below
// 1e-14 max|H_a| and v_{a+1} exists, factors Hbar instead (a rotations,
// least squares).  Writes R, rot (c, s pairs), rinv (reciprocal pivots, 0 for
// a zero pivot) and returns lsq / nrot.
__device__ __forceinline__ void factor_hessenberg(const double* Hb, int ld, int a, int has_next,
                                                  double* R, double* rot, double* rinv,
                                                  int* lsq_out, int* nrot_out) {
  double hmax = 0.0;
  for (int j = 0; j < a; ++j)
    for (int i = 0; i < a && i <= j + 1; ++i) hmax = fmax(hmax, fabs(Hb[i + j * ld]));
  int lsq = 0, nrot = 0;
  for (int pass = 0; pass < 2; ++pass) {
    lsq = pass;
    const int nr = lsq ? a + 1 : a;
    for (int j = 0; j < a; ++j)
      for (int i = 0; i <= a; ++i) R[i + j * ld] = (i < nr && i <= j + 1) ? Hb[i + j * ld] : 0.0;
    nrot = 0;
    for (int j = 0; j < a && j + 1 < nr; ++j) {
      double c, s;
      givens_rot(R[j + j * ld], R[(j + 1) + j * ld], c, s);
      for (int l = j; l < a; ++l) {
        const double t1 = R[j + l * ld], t2 = R[(j + 1) + l * ld];
        R[j + l * ld] = c * t1 + s * t2;
        R[(j + 1) + l * ld] = -s * t1 + c * t2;
      }
      rot[2 * j] = c;
      rot[2 * j + 1] = s;
      ++nrot;
    }
    int singular = 0;
    for (int j = 0; j < a; ++j)
      if (!(fabs(R[j + j * ld]) > 1e-14 * hmax)) singular = 1;
    if (singular && !lsq && has_next) continue;
    break;
  }
  for (int j = 0; j < a; ++j) rinv[j] = (R[j + j * ld] != 0.0) ? 1.0 / R[j + j * ld] : 0.0;
  *lsq_out = lsq;
  *nrot_out = nrot;
}

// alpha from c in place, c <- R^{-1} (G c), by one warp: the rotations on lane
// 0, then a column-oriented back substitution (lane l owns rows l, l+32).
// c lives in shared memory; a <= 64.  Ends with __syncwarp.
__device__ __forceinline__ void solve_projected_warp(double* c, int a, int nrot, const double* R,
                                                     int ld, const double* rot,
                                                     const double* rinv, int lane) {
  if (lane == 0) {
    for (int j = 0; j < nrot; ++j) {
      const double cc = rot[2 * j], s = rot[2 * j + 1];
      const double t1 = c[j], t2 = c[j + 1];
      c[j] = cc * t1 + s * t2;
      c[j + 1] = -s * t1 + cc * t2;
    }
  }
  __syncwarp();
  double g0 = (lane < a) ? c[lane] : 0.0;
  double g1 = (lane + 32 < a) ? c[lane + 32] : 0.0;
  __syncwarp();
  for (int i = a - 1; i >= 0; --i) {
    const double gi = __shfl_sync(0xffffffffu, i < 32 ? g0 : g1, i & 31);
    const double ai = gi * rinv[i];
    if (lane == 0) c[i] = ai;
    if (lane < i) g0 = fma(-R[lane + i * ld], ai, g0);
    if (lane + 32 < i) g1 = fma(-R[(lane + 32) + i * ld], ai, g1);
  }
  __syncwarp();
}

// One tile of the tensor-core projection GEMM: targets row0..row0+127 of the
// BF16 right-hand-side matrix against basis rows vrow0..vrow0+47; C rows
// crow0 + (0..count), columns 0..nv.
struct ProjTile {
  int row0, vrow0, crow0, count, nv;
  int ccol0;        // first C column of this tile
  int kc0, kc1;     // K range in 64-element chunks; kc1 == 0: the whole K
  int atomic;       // accumulate into C with atomicAdd (split K) instead of storing
};

// Launchers (defined in the .cu files; return a cudaError_t of the launch).
cudaError_t launch_gmres_fp64(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                              cudaStream_t st);
// The same with the optional paths compiled in (exact Galerkin, Picard, score,
// explicit A_proj), and the BiCGSTAB seed solver.
cudaError_t launch_gmres_fp64_feat(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st);
cudaError_t launch_gmres_fp64_bicg(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                   cudaStream_t st);
cudaError_t launch_gmres_fp64_dense(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                    cudaStream_t st);
cudaError_t launch_gmres_fp64_score(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                    cudaStream_t st);
cudaError_t launch_gmres_fp64_picard(const GmresParams& p, int ept, int nt, int minb, size_t smem,
                                     cudaStream_t st);
size_t gmres_fp64_smem_bytes(int ept, int nt, int S, int m);
size_t gmres_mixed_smem_bytes(int ept, int nt, int S, int m);
cudaError_t launch_gmres_mixed(const GmresParams& p, int ept, int nt, size_t smem,
                               cudaStream_t st);
size_t gmres_cluster_smem_bytes(int ept, int nt, int S, int m);
// Cluster of cs CTAs per system (grids above 4096 unknowns, mixed precision).
cudaError_t launch_gmres_cluster(const GmresParams& p, int ept, int nt, int cs, int minb, size_t smem,
                                 cudaStream_t st);
// The N <= 1024 instantiation (4 points x 256 threads) on an explicit grid;
// the kernel strides over systems, block b using Krylov workspace slice b.
cudaError_t launch_gmres_fp64_1k_grid(const GmresParams& p, size_t smem, int grid,
                                      cudaStream_t st);
cudaError_t launch_apply(const SysDesc* sys, int nsys, int mode, cudaStream_t st);
cudaError_t launch_factor(const FactorParams& p, cudaStream_t st);
cudaError_t launch_project_fp64(const ProjParams& p, int ept, int nt, cudaStream_t st);
cudaError_t launch_advance(int* step, cudaStream_t st, int by = 1, int* zero = nullptr, int nzero = 1);

// Seed cycling (kp_cycle.cu): per timestep of a launch and per seed, the
// basis the seed serves its targets, written to separate output slots (the
// solver's slots keep each seed's own basis): a seed without predecessor
// serves its own slot as it is; a linked one serves its own basis vectors
// followed by those of its predecessors, newest first, orthonormalised (CGS2)
// and capped at max_a, with the explicit A_proj = V^T A_seed V (dense slot).
struct CycleParams {
  const SysDesc* sys;       // seed descriptors (H, W, h, dt, f), plan order
  const int* prev;          // [ns] predecessor of each plan seed, or -1
  int ns;
  const double* slotV;      // [slots][max_a + 1][ld] the seeds' own bases
  const SlotMeta* slotMeta;
  const double* slotR;      // [slots][(max_a + 1) * max_a]
  const double* slotM;      // [slots][ld] lagged field of each slot's seed solve
  double* outV;             // served bases, same layout
  SlotMeta* outMeta;
  double* outR;
  int max_a, ld;
  const int* step;          // timesteps *step + step_offset .. + win - 1, below step_end
  int step_offset, win;
  const int* step_end;
  const double* g2_sched;
  double b_scale;           // the solvers' right-hand-side scale: A_proj of A / b_scale
  int slot_sets;            // slot of seed s at t: (t mod slot_sets) * ns + s
  float* scratch;           // [gridDim.x][max_a][ld] FP32 kept vectors
};
constexpr int kCycleThreads = 256;
constexpr int kCycleMaxN = 4096;
cudaError_t launch_cycle(const CycleParams& p, int nmax, int grid, cudaStream_t st);   // nmax: largest seed grid

// 3x3 convolutions on the tensor cores (kp_conv_tc.cu): padded-column BF16
// activation layout [B][chunks of 8 channels][Rp rows][8], pixel (i, j) at row
// halo + i*(H+2) + 1 + j, zero rows elsewhere.
struct ConvGeom { int H, W, halo, nst, Rp; };
ConvGeom conv_geom(int H, int W);
size_t conv_smem_bytes(const ConvGeom& g, int cic, int nout);
cudaError_t launch_conv_weights(const float* Wl, int cin, int cout, int cic, int nout, __nv_bfloat16* wf,
                                cudaStream_t st);
cudaError_t launch_planes_to_padded(const float* X, int B, int C, int chunks, const ConvGeom& g,
                                    __nv_bfloat16* out, cudaStream_t st);
cudaError_t launch_conv3x3(const __nv_bfloat16* in, int B, int cic, const __nv_bfloat16* wf, const float* bias,
                           int cout, int nout, const ConvGeom& g, __nv_bfloat16* out_pad, float* out_f32,
                           int* err, int sms, cudaStream_t st);
// Resident blocks per SM of the FP64 solver shape (0 if unknown).
int gmres_fp64_blocks_per_sm(int ept, int nt, int minb, size_t smem);
// dst[q] = src[perm[q]] (gather) or dst[perm[q]] = src[q] (scatter), planes of n doubles
cudaError_t launch_permute(double* dst, const double* src, const int* perm, int count, int n,
                           int gather, cudaStream_t st);
// b16[q] = bf16(src[q] * scale), planes of n doubles into rows of ld BF16
cudaError_t launch_to_bf16(__nv_bfloat16* dst, int ld, const double* src, int count, int n,
                           double scale, cudaStream_t st);
size_t proj_gemm_smem_bytes();
// Tensor map of a row-major BF16 matrix (rows x cols, row stride ld elements)
// read in boxes of box_rows x 64 with 128-byte swizzle.
cudaError_t make_bf16_map(void* map, const void* base, int rows, int cols, int ld, int box_rows);
// Target Gram matrices of exact Galerkin projection in mixed precision
// (kp_gram.cu): per timestep, the product rows P and G0 of every seed basis of
// the timestep's slot set, and the coefficient rows Q of every target; the
// GEMM C = Q P^T runs on launch_proj_gemm_bf16.
struct GramParams {
  const SysDesc* seeds;       // [ns] grid of each seed (slot index within the set)
  const SysDesc* targets;     // [nt]
  int ns, nt;
  int A;                      // Gram dimension bound (pairs p * A + q)
  int max_a, slot_ld, max_n;
  const int* step;            // current target timestep (device counter)
  const double* g2_sched;
  double b_scale;
  const SlotMeta* slotMeta;
  const float* slotV32;
  __nv_bfloat16* Pb;          // [2 ns A^2][p_ld] rows v_p o Dx v_q | v_p o Dy v_q
  int p_ld;
  float* G0;                  // [2 ns][A^2]
  __nv_bfloat16* Qb;          // [nt][q_ld] rows qx_i | qy_i
  int q_ld;
};
cudaError_t launch_gram_products(const GramParams& gp, cudaStream_t st);
cudaError_t launch_gram_coeff(const GramParams& gp, cudaStream_t st);

cudaError_t launch_proj_gemm_bf16(const CUtensorMap& mapB, const CUtensorMap& mapV,
                                  const ProjTile* tiles, int ntiles, int K, float* C, int ldc,
                                  int* err, int grid, cudaStream_t st);
cudaError_t launch_widen(const float* src, size_t src_ld, double* dst, size_t dst_ld, int n, int rows,
                         cudaStream_t st);

}  // namespace kp
