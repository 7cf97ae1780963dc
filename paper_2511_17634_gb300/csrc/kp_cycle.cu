// kp_cycle.cu -- seed cycling with subspace expansion.  Sec. 5.2 takes a new
// seed every 50 images and caps the subspace at a = 20 vectors; the paragraph
// the source of Sec. 3 leaves commented out accumulates the key vectors of
// every new seed into an increasingly rich basis.  A seed with a predecessor
// serves its targets the basis built from its own basis vectors first, then
// the predecessor's served ones, each orthogonalised twice (CGS2) against
// those kept and kept if more than 1e-10 of its norm remains, up to max_a; so
// the newest seed's space is always whole.  A_proj = V^T A_seed V is formed
// with the seed's own operator (rebuilt from the lagged field its solve used)
// and served as a dense slot, which the targets solve by LU.
//
// Because every served basis keeps its first vectors and drops only its tail,
// the served basis of a seed is the first max_a directions of its own basis
// followed by its predecessors' own bases, newest first.  So each seed's
// basis is built from the own bases along its chain, independently of the
// others: one block per (timestep, seed), all in parallel, into separate
// output slots.  FP64.
#include "kp_internal.cuh"

namespace kp {
namespace {

// EPT points per thread: 4 for grids of <= 1024 points, 16 up to 4096
template <int kEPT>
__global__ void __launch_bounds__(kCycleThreads) cycle_kernel(const CycleParams p) {
  constexpr int NT = kCycleThreads;
  __shared__ double red[(NT / 32) * kMaxV];
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
  // block sums of nv values fn(i) into hb[0..nv)
  auto reduce = [&](int nv, auto&& fn) {
    block_partials<NT>(nv, fn, red);
    if (warp == 0)
      for (int i = lane; i < nv; i += 32) hb[i] = cross_warp<NT>(red, i);
    __syncthreads();
  };
  double w[kEPT];
  int cnt = 0;
  auto keep = [&](const double* u) {
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int pp = tid + k * NT;
      w[k] = pp < N ? u[pp] : 0.0;
    }
    // two passes, each one batched reduction of <v_i, w> and ||w||^2; after
    // the second, ||w_2||^2 = ||w_1||^2 - ||h_2||^2 (h_2 = O(eps))
    double n0 = 0.0, n1 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      reduce(cnt + 1, [&](int i) {
        double acc = 0.0;
        if (i < cnt) {
          const double* vi = Vo + (size_t)i * p.ld;
#pragma unroll
          for (int k = 0; k < kEPT; ++k) {
            const int pp = tid + k * NT;
            if (pp < N) acc = fma(vi[pp], w[k], acc);
          }
        } else {
#pragma unroll
          for (int k = 0; k < kEPT; ++k) acc = fma(w[k], w[k], acc);
        }
        return acc;
      });
      double hh2 = 0.0;
      for (int i = 0; i < cnt; ++i) {
        const double hi = hb[i];
        hh2 = fma(hi, hi, hh2);
        const double* vi = Vo + (size_t)i * p.ld;
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
          const int pp = tid + k * NT;
          if (pp < N) w[k] = fma(-hi, vi[pp], w[k]);
        }
      }
      if (pass == 0) {
        n0 = hb[cnt];
      } else if (hh2 <= 0.25 * hb[cnt]) {
        n1 = hb[cnt] - hh2;
      } else {                                 // large correction: recompute the norm
        reduce(1, [&](int) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < kEPT; ++k) acc = fma(w[k], w[k], acc);
          return acc;
        });
        n1 = hb[0];
      }
    }
    if (!(n1 > 1e-20 * n0)) return;            // no new direction (norm ratio 1e-10)
    const double inv = 1.0 / sqrt(n1);
    double* vn = Vo + (size_t)cnt * p.ld;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int pp = tid + k * NT;
      if (pp < N) vn[pp] = w[k] * inv;
    }
    ++cnt;
  };
  // own basis (orthonormal already: copied), then the predecessors' own
  // bases, newest first, until full
  {
    const int na = min(ms.a, p.max_a);
    const double* Vs = p.slotV + (size_t)ss * vstride;
    for (int e = tid; e < na * p.ld; e += NT) Vo[e] = Vs[e];
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
  // right-hand-side scale as the solvers apply it
  const double* mt = p.slotM + (size_t)ss * p.ld;
  const double hh = d.h;
  const double g2 = p.g2_sched[t];
  const double osc = p.b_scale != 0.0 ? 1.0 / p.b_scale : 1.0;
  const double cc = g2 / (2.0 * hh * hh) * osc;
  const double ee = g2 / (8.0 * hh * hh) * osc;
  const double cd = (1.0 / d.dt + 2.0 * g2 / (hh * hh)) * osc;
  const double i2h = osc / (2.0 * hh);
  double* R = p.outR + (size_t)ss * rstride;
  for (int kc = 0; kc < cnt; ++kc) {
    const double* v = Vo + (size_t)kc * p.ld;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int pp = tid + k * NT;
      w[k] = 0.0;
      if (pp < N) {
        const int i = pp / H, jj = pp - i * H;
        const double mE = (i + 1 < W) ? mt[pp + H] : 0.0;
        const double mW = (i > 0) ? mt[pp - H] : 0.0;
        const double mN = (jj + 1 < H) ? mt[pp + 1] : 0.0;
        const double mS = (jj > 0) ? mt[pp - 1] : 0.0;
        const double fxp = d.fx ? d.fx[pp] : 0.0;
        const double fyp = d.fy ? d.fy[pp] : 0.0;
        const double dmx = mE - mW, dmy = mN - mS;
        double y = cd * v[pp];
        if (i + 1 < W) y = fma(-cc + fxp * i2h - ee * dmx, v[pp + H], y);
        if (i > 0) y = fma(-cc - fxp * i2h + ee * dmx, v[pp - H], y);
        if (jj + 1 < H) y = fma(-cc + fyp * i2h - ee * dmy, v[pp + 1], y);
        if (jj > 0) y = fma(-cc - fyp * i2h + ee * dmy, v[pp - 1], y);
        w[k] = y;
      }
    }
    reduce(cnt, [&](int l) {
      const double* vl = Vo + (size_t)l * p.ld;
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < kEPT; ++k) {
        const int pp = tid + k * NT;
        if (pp < N) acc = fma(vl[pp], w[k], acc);
      }
      return acc;
    });
    for (int l = tid; l < cnt; l += NT) R[l + (size_t)kc * (p.max_a + 1)] = hb[l];
  }
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
