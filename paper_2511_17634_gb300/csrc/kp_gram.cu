// kp_gram.cu -- the target Gram matrices of exact Galerkin projection in mixed
// precision (Sec. 3, Phase 2 with each target's own operator instead of the
// seed-matrix shortcut: G_i = V_a^T A_i V_a, G_i alpha = V_a^T b_i,
// x0 = V_a alpha), with the target-dependent part on the tensor cores.
//
// The operator of target i at a timestep (the Sec. 2.3 coefficients, divided
// by the right-hand-side scale as the solvers apply them) is
//   A_i v = cd v - c S v + qx_i o Dx v + qy_i o Dy v,
//   S v = v_E + v_W + v_N + v_S,  Dx v = v_E - v_W,  Dy v = v_N - v_S
// (neighbours outside the grid are zero), and only qx_i, qy_i -- built from the
// target's lagged field -- depend on the target.  Hence, for basis vectors
// v_p, v_q of the seed,
//   G_i[p][q] = G0[p][q] + sum_k qx_i[k] Px_pq[k] + sum_k qy_i[k] Py_pq[k],
//   G0[p][q] = cd v_p.v_q - c v_p.(S v_q),  Px_pq = v_p o Dx v_q,  Py_pq = v_p o Dy v_q.
// G0 and the products P belong to the seed basis (gram_products_kernel, per
// timestep and seed); the sums for all targets of a seed are one GEMM
//   C[i][(p,q)] = Q_i . P_(p,q),   Q_i = [qx_i | qy_i]   (K = 2N),
// BF16 operands with FP32 accumulation on tcgen05 (kp_proj_tc.cu), so the
// per-target work is a row of coefficients instead of a stencil applications
// and a^2 dot products.  The solver adds G0 + C, solves by LU and projects.
#include <cuda_bf16.h>

#include "kp_dd.cuh"
#include "kp_internal.cuh"

namespace kp {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramEPT = 16;            // points per thread: grids up to 4096 points

// Block (seed slot s of the current timestep's set, basis column q): the
// product rows (p, q) for every p < A and G0[p][q].  Rows and entries with p or
// q at or past the slot's a (or a slot of another timestep) are zeros.
__global__ void __launch_bounds__(kGramThreads) gram_products_kernel(GramParams gp) {
  constexpr int NT = kGramThreads;
  __shared__ float red[2][kMaxV][NT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int A = gp.A;
  const int si = blockIdx.x / A, q = blockIdx.x - si * A;
  const int t = *gp.step;
  const int slot = (t % 2) * gp.ns + si;
  const SysDesc d = gp.seeds[si];
  const int H = d.H, W = d.W, N = H * W;
  const SlotMeta mt = gp.slotMeta[slot];
  const bool live = mt.timestep == t && mt.N == N && q < mt.a;
  const int a = live ? min(mt.a, A) : 0;
  const double g2 = gp.g2_sched[t];
  const double osc = 1.0 / gp.b_scale;
  const double hh = d.h;
  const float cc = (float)(g2 / (2.0 * hh * hh) * osc);
  const float cd = (float)((1.0 / d.dt + 2.0 * g2 / (hh * hh)) * osc);
  const float* V = gp.slotV32 + (size_t)slot * (gp.max_a + 1) * gp.slot_ld;
  const float* vq = V + (size_t)q * gp.slot_ld;
  float dx[kGramEPT], dy[kGramEPT], sv[kGramEPT], qv[kGramEPT];
#pragma unroll
  for (int k = 0; k < kGramEPT; ++k) {
    const int pp = tid + k * NT;
    dx[k] = dy[k] = sv[k] = qv[k] = 0.f;
    if (live && pp < N) {
      const int i = pp / H, j = pp - i * H;
      const float vE = i + 1 < W ? vq[pp + H] : 0.f, vW = i > 0 ? vq[pp - H] : 0.f;
      const float vN = j + 1 < H ? vq[pp + 1] : 0.f, vS = j > 0 ? vq[pp - 1] : 0.f;
      dx[k] = vE - vW;
      dy[k] = vN - vS;
      sv[k] = vE + vW + vN + vS;
      qv[k] = vq[pp];
    }
  }
  for (int p = 0; p < A; ++p) {
    __nv_bfloat16* row = gp.Pb + ((size_t)slot * A * A + (size_t)p * A + q) * gp.p_ld;
    const float* vp = V + (size_t)p * gp.slot_ld;
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int k = 0; k < kGramEPT; ++k) {
      const int pp = tid + k * NT;
      if (pp < N) {
        const float v = p < a ? vp[pp] : 0.f;
        row[pp] = __float2bfloat16_rn(v * dx[k]);
        row[N + pp] = __float2bfloat16_rn(v * dy[k]);
        s1 = fmaf(v, qv[k], s1);
        s2 = fmaf(v, sv[k], s2);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      red[0][p][warp] = s1;
      red[1][p][warp] = s2;
    }
  }
  __syncthreads();
  for (int p = tid; p < A; p += NT) {
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
      s1 += red[0][p][w];
      s2 += red[1][p][w];
    }
    gp.G0[(size_t)slot * A * A + (size_t)p * A + q] = cd * s1 - cc * s2;
  }
}

// Block per target i of the current timestep: Q_i = [qx_i | qy_i] in BF16,
// qx = f_x / (2h) - e (m_E - m_W), qy likewise, from the target's lagged field
// (its FP64 values truncated to FP32 without FP64 instructions; BF16 keeps 8
// bits of them anyway).
__global__ void __launch_bounds__(kGramThreads) gram_coeff_kernel(GramParams gp) {
  const int i = blockIdx.x;
  const SysDesc d = gp.targets[i];
  const int H = d.H, W = d.W, N = H * W;
  const double g2 = gp.g2_sched[*gp.step];
  const double osc = 1.0 / gp.b_scale;
  const float ee = (float)(g2 / (8.0 * d.h * d.h) * osc);
  const float i2h = (float)(osc / (2.0 * d.h));
  __nv_bfloat16* row = gp.Qb + (size_t)i * gp.q_ld;
  for (int pp = threadIdx.x; pp < N; pp += blockDim.x) {
    const int x = pp / H, y = pp - x * H;
    const float mE = x + 1 < W ? dd_from_double(d.mt[pp + H]).hi : 0.f;
    const float mW = x > 0 ? dd_from_double(d.mt[pp - H]).hi : 0.f;
    const float mN = y + 1 < H ? dd_from_double(d.mt[pp + 1]).hi : 0.f;
    const float mS = y > 0 ? dd_from_double(d.mt[pp - 1]).hi : 0.f;
    float qx = -ee * (mE - mW), qy = -ee * (mN - mS);
    if (d.fx) qx = fmaf(dd_from_double(d.fx[pp]).hi, i2h, qx);
    if (d.fy) qy = fmaf(dd_from_double(d.fy[pp]).hi, i2h, qy);
    row[pp] = __float2bfloat16_rn(qx);
    row[N + pp] = __float2bfloat16_rn(qy);
  }
}

}  // namespace

cudaError_t launch_gram_products(const GramParams& gp, cudaStream_t st) {
  if (gp.ns <= 0 || gp.A <= 0) return cudaSuccess;
  if (gp.A > kMaxV || gp.max_n > kGramEPT * kGramThreads) return cudaErrorInvalidValue;
  gram_products_kernel<<<gp.ns * gp.A, kGramThreads, 0, st>>>(gp);
  return cudaGetLastError();
}

cudaError_t launch_gram_coeff(const GramParams& gp, cudaStream_t st) {
  if (gp.nt <= 0) return cudaSuccess;
  gram_coeff_kernel<<<gp.nt, kGramThreads, 0, st>>>(gp);
  return cudaGetLastError();
}

}  // namespace kp
