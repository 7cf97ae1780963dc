// kp_cycle.cu -- seed cycling with subspace expansion.  Sec. 5.2 takes a new
// seed every 50 images and caps the subspace at a = 20 vectors; the paragraph
// the source of Sec. 3 leaves commented out accumulates the key vectors of
// every new seed into an increasingly rich basis.  A seed with a predecessor
// serves its targets the basis built from its own basis vectors first, then
// the predecessor's served ones, each orthogonalised twice (CGS2) against
// those kept and kept while a new direction remains, up to max_a; so the
// newest seed's space is always whole.  A_proj = V^T A_seed V is formed with
// the seed's own operator (rebuilt from the lagged field its solve used) and
// served as a dense slot, which the targets solve by LU.
//
// Because every served basis keeps its first vectors and drops only its tail,
// the served basis of a seed is the first max_a directions of its own basis
// followed by its predecessors' own bases, newest first.  So each seed's
// basis is built from the own bases along its chain, independently of the
// others: one block per (timestep, seed), all in parallel, into separate
// output slots.
//
// Precision: the served basis only forms the targets' starting guess (the
// FP64 refine and its true-residual test fix the accuracy), so it is built
// and A_proj formed in FP32 on the FP32 pipe -- 64x the FP64 rate of this
// part -- with FP64 sums across warps; a vector counts as a new direction if
// more than 1e-4 of its norm remains after the two passes (FP32 resolves no
// less; the FP64 definition uses 1e-10).  The served vectors are stored as
// FP64, orthonormal to FP32 accuracy.
#include "kp_internal.cuh"

namespace kp {
namespace {

// EPT points per thread: 4 for grids of <= 1024 points, 16 up to 4096
template <int kEPT>
__global__ void __launch_bounds__(kCycleThreads) cycle_kernel(const CycleParams p) {
  constexpr int NT = kCycleThreads;
  __shared__ float red32[(NT / 32) * kMaxV];
  __shared__ double hb[kMaxV];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t0 = *p.step + p.step_offset;
  const int nstep = min(p.win > 0 ? p.win : 1, *p.step_end - t0);
  const int kstep = blockIdx.x / p.ns, s = blockIdx.x - kstep * p.ns;
  if (kstep >= nstep) return;
  const int t = t0 + kstep;
  const int sets = p.slot_sets > 2 ? p.slot_sets : 2;
  const int pb = (t % sets) * p.ns;
  const int ss = pb + s;
  const size_t vstride = (size_t)(p.max_a + 1) * p.ld;
  const size_t rstride = (size_t)(p.max_a + 1) * p.max_a;
  const SlotMeta ms = p.slotMeta[ss];
  double* Vo = p.outV + (size_t)ss * vstride;
  if (p.prev[s] < 0 || ms.timestep != t) {
    // served as it is: copy basis, factor and metadata
    const int nv = ms.timestep == t ? ms.a + ms.has_next : 0;
    const double* Vs = p.slotV + (size_t)ss * vstride;
    for (int e = tid; e < nv * p.ld; e += NT) Vo[e] = Vs[e];
    const double* Rs = p.slotR + (size_t)ss * rstride;
    double* Ro = p.outR + (size_t)ss * rstride;
    const int nr = ms.timestep == t ? (p.max_a + 1) * min(ms.a, p.max_a) : 0;   // a columns
    for (int e = tid; e < nr; e += NT) Ro[e] = Rs[e];
    if (tid == 0) p.outMeta[ss] = ms;
    return;
  }
  const SysDesc d = p.sys[s];
  const int H = d.H, W = d.W, N = H * W;
  float* Ws = p.scratch + (size_t)blockIdx.x * p.max_a * p.ld;   // kept vectors, FP32
  // block sums of nv FP32 values fn(i) into hb[0..nv) (FP64 results)
  auto reduce = [&](int nv, auto&& fn) {
    block_partials_f32x<NT>(nv, fn, red32);
    if (warp == 0) cross_warp_f32<NT>(red32, nv, hb, lane);
    __syncthreads();
  };
  float w[kEPT];
  int cnt = 0;
  auto keep = [&](const double* u) {
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int pp = tid + k * NT;
      w[k] = pp < N ? (float)u[pp] : 0.f;
    }
    // two passes, each one batched reduction of <v_i, w> and ||w||^2; after
    // the second, ||w_2||^2 = ||w_1||^2 - ||h_2||^2 unless it removed a lot
    double n0 = 0.0, n1 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      reduce(cnt + 1, [&](int i) {
        float acc = 0.f;
        if (i < cnt) {
          const float* vi = Ws + (size_t)i * p.ld;
#pragma unroll
          for (int k = 0; k < kEPT; ++k) {
            const int pp = tid + k * NT;
            if (pp < N) acc = fmaf(vi[pp], w[k], acc);
          }
        } else {
#pragma unroll
          for (int k = 0; k < kEPT; ++k) acc = fmaf(w[k], w[k], acc);
        }
        return acc;
      });
      double hh2 = 0.0;
      for (int i = 0; i < cnt; ++i) {
        const double hi = hb[i];
        hh2 += hi * hi;
        const float hf = (float)hi;
        const float* vi = Ws + (size_t)i * p.ld;
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
          const int pp = tid + k * NT;
          if (pp < N) w[k] = fmaf(-hf, vi[pp], w[k]);
        }
      }
      if (pass == 0) {
        n0 = hb[cnt];
      } else if (hh2 <= 0.25 * hb[cnt]) {
        n1 = hb[cnt] - hh2;
      } else {                                 // large correction: recompute the norm
        reduce(1, [&](int) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < kEPT; ++k) acc = fmaf(w[k], w[k], acc);
          return acc;
        });
        n1 = hb[0];
      }
    }
    // a new direction keeps more than 1e-4 of its norm (FP32 resolves no less)
    if (!(n1 > 1e-8 * n0)) return;
    const float inv = (float)(1.0 / sqrt(n1));
    float* vn = Ws + (size_t)cnt * p.ld;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int pp = tid + k * NT;
      if (pp < N) vn[pp] = w[k] * inv;
    }
    ++cnt;
  };
  // own basis (orthonormal already: taken as it is), then the predecessors'
  // own bases, newest first, until full
  {
    const int na = min(ms.a, p.max_a);
    const double* Vs = p.slotV + (size_t)ss * vstride;
    for (int kc = 0; kc < na; ++kc)
      for (int pp = tid; pp < N; pp += NT) Ws[(size_t)kc * p.ld + pp] = (float)Vs[(size_t)kc * p.ld + pp];
    cnt = na;
    __syncthreads();
  }
  for (int u = p.prev[s], depth = 0; u >= 0 && cnt < p.max_a && depth < p.ns; u = p.prev[u], ++depth) {
    const SlotMeta mu = p.slotMeta[pb + u];
    if (mu.timestep != t || mu.N != N) break;  // uniform
    const double* Vu = p.slotV + (size_t)(pb + u) * vstride;
    for (int k = 0; k < mu.a && cnt < p.max_a; ++k) keep(Vu + (size_t)k * p.ld);
  }
  __syncthreads();                             // kept vectors complete for the stencil

  // A_proj = V^T A_s V with the seed's operator (Sec. 2.3 coefficients from
  // the lagged field of its solve, zero outside the grid), divided by the
  // right-hand-side scale as the solvers apply it:
  //   A v = cd v - c (v_E + v_W + v_N + v_S) + q_x (v_E - v_W) + q_y (v_N - v_S)
  const double* mt = p.slotM + (size_t)ss * p.ld;
  const double hh = d.h;
  const double g2 = p.g2_sched[t];
  const double osc = p.b_scale != 0.0 ? 1.0 / p.b_scale : 1.0;
  const double cc = g2 / (2.0 * hh * hh) * osc;
  const double ee = g2 / (8.0 * hh * hh) * osc;
  const double cd = (1.0 / d.dt + 2.0 * g2 / (hh * hh)) * osc;
  const double i2h = osc / (2.0 * hh);
  const float ccf = (float)cc, cdf = (float)cd;
  float qx[kEPT], qy[kEPT];
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int pp = tid + k * NT;
    qx[k] = qy[k] = 0.f;
    if (pp < N) {
      const int i = pp / H, jj = pp - i * H;
      const double mE = (i + 1 < W) ? mt[pp + H] : 0.0;
      const double mW = (i > 0) ? mt[pp - H] : 0.0;
      const double mN = (jj + 1 < H) ? mt[pp + 1] : 0.0;
      const double mS = (jj > 0) ? mt[pp - 1] : 0.0;
      const double fxp = d.fx ? d.fx[pp] : 0.0;
      const double fyp = d.fy ? d.fy[pp] : 0.0;
      qx[k] = (float)(fxp * i2h - ee * (mE - mW));
      qy[k] = (float)(fyp * i2h - ee * (mN - mS));
    }
  }
  double* R = p.outR + (size_t)ss * rstride;
  for (int kc = 0; kc < cnt; ++kc) {
    const float* v = Ws + (size_t)kc * p.ld;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int pp = tid + k * NT;
      w[k] = 0.f;
      if (pp < N) {
        const int i = pp / H, jj = pp - i * H;
        const float vE = (i + 1 < W) ? v[pp + H] : 0.f;
        const float vW = (i > 0) ? v[pp - H] : 0.f;
        const float vN = (jj + 1 < H) ? v[pp + 1] : 0.f;
        const float vS = (jj > 0) ? v[pp - 1] : 0.f;
        w[k] = cdf * v[pp] - ccf * (vE + vW + vN + vS) + qx[k] * (vE - vW) + qy[k] * (vN - vS);
      }
    }
    reduce(cnt, [&](int l) {
      const float* vl = Ws + (size_t)l * p.ld;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < kEPT; ++k) {
        const int pp = tid + k * NT;
        if (pp < N) acc = fmaf(vl[pp], w[k], acc);
      }
      return acc;
    });
    for (int l = tid; l < cnt; l += NT) R[l + (size_t)kc * (p.max_a + 1)] = hb[l];
  }
  // the served basis, as FP64
  for (int kc = 0; kc < cnt; ++kc)
    for (int pp = tid; pp < N; pp += NT) Vo[(size_t)kc * p.ld + pp] = (double)Ws[(size_t)kc * p.ld + pp];
  if (tid == 0) {
    SlotMeta mo;
    mo.a = cnt;
    mo.has_next = 0;
    mo.timestep = t;
    mo.N = N;
    mo.lsq = 0;
    mo.nrot = 0;
    mo.dense = 1;
    mo.pad_ = 0;
    p.outMeta[ss] = mo;
  }
}

}  // namespace

cudaError_t launch_cycle(const CycleParams& p, int nmax, int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  if (nmax <= 4 * kCycleThreads) cycle_kernel<4><<<grid, kCycleThreads, 0, st>>>(p);
  else cycle_kernel<kCycleMaxN / kCycleThreads><<<grid, kCycleThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace kp
