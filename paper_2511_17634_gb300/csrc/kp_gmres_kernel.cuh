// kp_gmres_kernel.cuh -- the FP64 batched GMRES(m) kernel template and its
// launcher, shared by kp_gmres.cu (the lean instantiations), kp_gmres_dense.cu
// (the projection through an explicit A_proj), kp_gmres_score.cu (the fused
// score / embedding output), kp_gmres_picard.cu (Picard iterations),
// kp_gmres_feat.cu (all of these and the exact-Galerkin initial guess) and
// kp_gmres_bicg.cu (BiCGSTAB seed solves).  The optional paths are compiled
// only into their variants, so the default solver keeps its registers for the
// hot loop; the variants compile in parallel.
//
// GB300 design notes (FP64 runs at 1/64 of the FP32 rate on this part, about
// 2 FP64 FMA per clock per SM, so FP64 instructions -- not HBM bytes -- bound
// this kernel):
//  * The operator is applied matrix-free.  Each thread keeps the four
//    off-diagonal coefficients of its EPT grid points in registers (computed
//    once per solve from the lagged field m~), the diagonal is a scalar, and
//    out-of-grid neighbours get a zero coefficient and a clamped index, so the
//    stencil is 1 MUL + 4 FMA per point with no branches.
//  * Krylov vectors v_0..v_{S-1} live in shared memory; the stencil reads its
//    neighbours there.  Vectors beyond S go to a per-block device workspace.
//  * Orthogonalisation is classical Gram-Schmidt applied twice (CGS2): every
//    pass is one batched reduction of all <v_i, w> at once instead of j
//    sequential reductions.  Reductions are warp reduce-scatter butterflies
//    over 8 values (about one FP64 add per value per lane instead of five)
//    followed by one cross-warp sum.
//  * Hessenberg, Givens rotations and the least-squares solve stay in FP64 on
//    one lane; the true residual b - A x is recomputed in FP64 at every restart.
#pragma once

#include "kp_internal.cuh"

namespace kp {
namespace {

struct Smem {
  double* V;     // [S][npad]
  double* xs;    // [npad]
  double* red;   // [NWARPS][kMaxV]
  double* hb;    // [kMaxV]
  double* Hr;    // [(m+1) * m] rotated Hessenberg, column-major, ld m+1
  double* g;     // [m+1]
  double* cs;    // [m]
  double* sn;    // [m]
  double* y;     // [m]
  double* rinv;  // [m] reciprocal pivots of the rotated Hessenberg
  double* sc;    // [8] scalars
  int* fl;       // [8] flags
};

__device__ __forceinline__ Smem carve(double* base, int S, int npad, int nwarps, int m) {
  Smem s;
  s.V = base;
  s.xs = s.V + (size_t)S * npad;
  s.red = s.xs + npad;
  s.hb = s.red + nwarps * kMaxV;
  s.Hr = s.hb + kMaxV;
  s.g = s.Hr + (m + 1) * m;
  s.cs = s.g + (m + 1);
  s.sn = s.cs + m;
  s.y = s.sn + m;
  s.rinv = s.y + m;
  s.sc = s.rinv + m;
  s.fl = reinterpret_cast<int*>(s.sc + 8);
  return s;
}

// VAR selects the code compiled into an instantiation: kVarLean (the plain
// solver), kVarDense (plus the projection through an explicit A_proj, for
// BiCGSTAB and cycled seed bases), kVarScore (plus the score / embedding
// epilogue), kVarPicard (plus Picard iterations), kVarFeat (all of these and
// exact Galerkin), kVarBicg (BiCGSTAB seed solves).
enum { kVarLean = 0, kVarFeat = 1, kVarBicg = 2, kVarDense = 3, kVarScore = 4, kVarPicard = 5 };

template <int EPT, int NT, int MINB, int VAR>
__global__ void __launch_bounds__(NT, MINB) gmres_fp64_kernel(const GmresParams p) {
  constexpr bool FEAT = VAR == kVarFeat;
  constexpr bool BICG = VAR == kVarBicg;
  constexpr bool DENSE = VAR == kVarFeat || VAR == kVarDense;
  constexpr bool SCORE = VAR == kVarFeat || VAR == kVarScore;
  constexpr bool PICARD = VAR == kVarFeat || VAR == kVarPicard;
  constexpr int NWARPS = NT / 32;
  extern __shared__ __align__(16) double smem_raw[];
  const int npad = EPT * NT;
  const int m = p.m;
  const int ld = m + 1;
  Smem sm = carve(smem_raw, p.S, npad, NWARPS, m);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* spill = p.spill ? p.spill + (size_t)blockIdx.x * (m + 1 - p.S) * npad : nullptr;
  auto slot = [&](int i) -> double* {
    return i < p.S ? sm.V + (size_t)i * npad : spill + (size_t)(i - p.S) * npad;
  };
  if (p.pdl & 1) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // timesteps of this launch (time march): t0 .. t0 + nstep - 1
  int t0 = 0, nstep = 1;
  if (p.step) {
    t0 = *p.step + p.step_offset;
    nstep = min(p.win > 0 ? p.win : 1, *p.step_end - t0);
    if (nstep <= 0) {                        // pipelined seed step past the run: nothing to do
      if (p.pdl & 2) asm volatile("griddepcontrol.wait;" ::: "memory");
      return;
    }
  }
  const double bsc = p.b_scale;
  const int nitems = p.nsys * nstep;
  int sysi = blockIdx.x, kstep = 0;          // static schedule: a block marches its systems
  for (;;) {
    if (p.queue) {
      // dynamic schedule over (timestep, system) items, timestep-major: a
      // block that finishes early takes the next item instead of idling
      // until the slowest system of its wave is done
      if (tid == 0) sm.fl[6] = atomicAdd(p.queue, 1);
      __syncthreads();
      const int item = sm.fl[6];
      if (item >= nitems) break;
      kstep = item / p.nsys;
      sysi = item - kstep * p.nsys;
    } else if (sysi >= p.nsys) {
      break;
    }
    const int tstep = t0 + kstep;
    if (p.done) {
      // m^{n-1} of this system comes from its previous item, claimed earlier
      // by a block that is therefore running: wait for its release
      const int need = tstep - *p.run_start + p.wait_bias;
      const int limit = p.wait_limit > 0 ? p.wait_limit : kWaitLimit;
      if (tid == 0) {
        int it = 0;
        while (ld_acquire_gpu(p.done + sysi) < need) {
          if (++it > limit) { atomicOr(p.err, 2); break; }
          __nanosleep(256);
        }
      }
      __syncthreads();
      (void)ld_acquire_gpu(p.done + sysi);    // orders this thread's loads of m^{n-1}
    }
    const int parity_base = slot_set_base(p, tstep);
    const SysDesc d = p.sys_par[0] ? p.sys_par[(tstep + p.sys_shift) & 1][sysi] : p.sys[sysi];
    const int H = d.H, W = d.W, N = H * W;
    const double hh = d.h;
    const double g2 = p.step ? p.g2_sched[tstep] : d.g2;
    // the system is solved as (A / s) x = b / s with s = b_scale (the march's
    // 1/dt): the right-hand side is read as stored and the scale goes on the
    // four operator constants, once per solve
    const double osc = bsc != 0.0 ? 1.0 / bsc : 1.0;
    const double cc = g2 / (2.0 * hh * hh) * osc;
    const double ee = g2 / (8.0 * hh * hh) * osc;
    const double cd = (1.0 / d.dt + 2.0 * g2 / (hh * hh)) * osc;
    const double i2h = osc / (2.0 * hh);
    bool capture = p.capV != nullptr;          // first solve of the timestep only
    const int cidx = p.factor ? parity_base + sysi : sysi;   // capture record (or seed slot)
    double* capV = capture ? p.capV + (size_t)cidx * (p.cap_a + 1) * p.cap_ld : nullptr;
    double* capH = capture ? p.capH + (size_t)cidx * (p.cap_a + 1) * p.cap_a : nullptr;
    if (capture && p.capM) {                   // the slot's operator, for seed cycling
      double* cm = p.capM + (size_t)cidx * p.cap_ld;
      for (int pp = tid; pp < N; pp += NT) cm[pp] = d.mt[pp];
    }

    // stencil coefficients (Sec. 2.3, listing after Eq. 11) from the lagged
    // field m~ (m^{n-1}, or the latest Picard iterate); zero where the
    // neighbour lies outside the grid
    double cE[EPT], cW[EPT], cN[EPT], cS[EPT];
    const bool drift = d.fx != nullptr || d.fy != nullptr;
    // score output (end of Sec. 2.3) and probability-flow embedding (Sec. 4.1):
    // the central differences of the input m^{n-1} are the ones the lagged
    // coefficients need, so the score of m^{n-1} (timestep n-1 of the output)
    // and the embedding step x += -dt (g^{n-1})^2 / 2 grad m^{n-1} are written
    // from here; the last timestep of a run writes the score of its own
    // solution in the epilogue
    const bool score_on = SCORE && p.score_stride && d.score;
    const double s_i2h = SCORE ? 0.5 / hh : 0.0;
    double cei = 0.0;                            // the Euler factor times 1/(2h)
    double* sc_in = nullptr;                     // score of the input, timestep tstep - 1
    if (SCORE && score_on) {
      const double g2prev = p.step ? p.g2_sched[tstep > 0 ? tstep - 1 : 0] : d.g2;
      cei = -0.5 * d.dt * g2prev * s_i2h;        // (g^0)^2 taken as (g^1)^2
      if (tstep > 0) sc_in = d.score + (size_t)(tstep - 1) * p.score_stride;
    }
    auto score_in = [&](int pp, double dmx, double dmy) {
      if (sc_in) {
        sc_in[pp] = dmx * s_i2h;
        sc_in[N + pp] = dmy * s_i2h;
      }
      d.emb[pp] = fma(cei, dmx, d.emb[pp]);
      d.emb[N + pp] = fma(cei, dmy, d.emb[N + pp]);
    };
    auto set_coeffs = [&](const double* mtl, bool input) {
      if (!drift) {                              // f = 0 (the method's systems): two terms each
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          cE[k] = cW[k] = cN[k] = cS[k] = 0.0;
          if (pp < N) {
            const int i = pp / H, j = pp - i * H;
            const double mE = (i + 1 < W) ? mtl[pp + H] : 0.0;
            const double mW = (i > 0) ? mtl[pp - H] : 0.0;
            const double mN = (j + 1 < H) ? mtl[pp + 1] : 0.0;
            const double mS = (j > 0) ? mtl[pp - 1] : 0.0;
            const double dmx = mE - mW, dmy = mN - mS;
            if (SCORE && score_on && input) score_in(pp, dmx, dmy);
            if (i + 1 < W) cE[k] = fma(-ee, dmx, -cc);
            if (i > 0) cW[k] = fma(ee, dmx, -cc);
            if (j + 1 < H) cN[k] = fma(-ee, dmy, -cc);
            if (j > 0) cS[k] = fma(ee, dmy, -cc);
          }
        }
        return;
      }
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        cE[k] = cW[k] = cN[k] = cS[k] = 0.0;
        if (pp < N) {
          const int i = pp / H, j = pp - i * H;
          const double mE = (i + 1 < W) ? mtl[pp + H] : 0.0;
          const double mW = (i > 0) ? mtl[pp - H] : 0.0;
          const double mN = (j + 1 < H) ? mtl[pp + 1] : 0.0;
          const double mS = (j > 0) ? mtl[pp - 1] : 0.0;
          const double fxp = d.fx ? d.fx[pp] : 0.0;
          const double fyp = d.fy ? d.fy[pp] : 0.0;
          const double dmx = mE - mW, dmy = mN - mS;
          if (SCORE && score_on && input) score_in(pp, dmx, dmy);
          if (i + 1 < W) cE[k] = -cc + fxp * i2h - ee * dmx;
          if (i > 0) cW[k] = -cc - fxp * i2h + ee * dmx;
          if (j + 1 < H) cN[k] = -cc + fyp * i2h - ee * dmy;
          if (j > 0) cS[k] = -cc - fyp * i2h + ee * dmy;
        }
      }
    };
    set_coeffs(d.mt, true);
    // r = b - A v, the product chain started from b (one multiply, five fused
    // multiply-adds per point)
    auto residual_of = [&](const double* v, double (&out)[EPT]) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        if (pp < N) {
          const int pe = min(pp + H, N - 1), pw = max(pp - H, 0);
          const int pn = min(pp + 1, N - 1), ps = max(pp - 1, 0);
          double t = fma(-cd, v[pp], d.b[pp]);
          t = fma(-cE[k], v[pe], t);
          t = fma(-cW[k], v[pw], t);
          t = fma(-cN[k], v[pn], t);
          out[k] = fma(-cS[k], v[ps], t);
        } else {
          out[k] = 0.0;
        }
      }
    };
    // Arnoldi runs on the shifted operator A - cd I (the constant diagonal
    // removed): the same Krylov space, with H_A = H + cd I restored in the
    // Hessenberg column.  A ~ (1/dt) I + small, so A v_j is nearly parallel to
    // v_j and the unshifted Gram-Schmidt would cancel most of it.
    auto apply_off = [&](const double* v, double (&out)[EPT]) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        if (pp < N) {
          const int pe = min(pp + H, N - 1), pw = max(pp - H, 0);
          const int pn = min(pp + 1, N - 1), ps = max(pp - 1, 0);
          out[k] = cE[k] * v[pe] + cW[k] * v[pw] + cN[k] * v[pn] + cS[k] * v[ps];
        } else {
          out[k] = 0.0;
        }
      }
    };
    auto bval = [&](int pp) { return (pp < N) ? d.b[pp] : 0.0; };

    // initial guess -> shared memory
    unsigned long long proj_flops = 0;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      double x0 = 0.0;
      if (pp < N) {
        if (p.x0_mode == X0_READ) x0 = d.x[pp];
        else if (p.x0_mode == X0_WARM) x0 = d.mt[pp];
      }
      sm.xs[pp] = x0;
    }
    if (p.x0_mode == X0_PROJECT) {
      // Sec. 3, Phase 2: x0 = V_a H_a^{-1} V_a^T b with the seed's stored basis
      const int sl = d.slot + parity_base;
      const SlotMeta mt = p.slotMeta[sl];
      if (mt.timestep == tstep && mt.N == N && mt.a > 0) {            // uniform per block
        const int a = mt.a;
        const int nv = mt.lsq ? a + 1 : a;
        const double* V = p.slotV + (size_t)sl * (p.max_a + 1) * p.slot_ld;
        double bv[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          bv[k] = pp < N ? d.b[pp] : 0.0;
        }
        block_partials<NT>(nv, [&](int i) {
          const double* vi = V + (size_t)i * p.slot_ld;
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            if (pp < N) s += vi[pp] * bv[k];
          }
          return s;
        }, sm.red);
        if (warp == 0) {
          for (int i = lane; i < nv; i += 32) sm.hb[i] = cross_warp<NT>(sm.red, i);
          __syncwarp();
          const double* R = p.slotR + (size_t)sl * (p.max_a + 1) * p.max_a;
          if (DENSE && mt.dense) {
            // BiCGSTAB seed basis: A_proj alpha = c with the stored explicit
            // A_proj = V^T A_seed V, LU with partial pivoting on this warp
            bool ok = a * a <= (m + 1) * m;
            if (ok) {
              for (int e = lane; e < a * a; e += 32) {
                const int l = e % a, k = e / a;
                sm.Hr[l + k * a] = R[l + (size_t)k * (p.max_a + 1)];
              }
              __syncwarp();
              ok = lu_solve_warp(sm.Hr, a, sm.hb, lane);
            }
            if (!ok)
              for (int i = lane; i < a; i += 32) sm.hb[i] = 0.0;
          } else {
            const double* rot = p.slotRot + (size_t)sl * 3 * p.max_a;
            solve_projected_warp(sm.hb, a, mt.nrot, R, p.max_a + 1, rot, rot + 2 * p.max_a, lane);
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          if (pp < N) {
            double xv = 0.0;
            for (int i = 0; i < a; ++i) xv = fma(sm.hb[i], V[(size_t)i * p.slot_ld + pp], xv);
            sm.xs[pp] = xv;
          }
        }
        proj_flops = (unsigned long long)(2 * nv + 2 * a) * (unsigned long long)N;
      }
    }
    if (FEAT && p.x0_mode == X0_GALERKIN) {
      // Sec. 3, Phase 2 without the seed-matrix shortcut: G = V_a^T A_i V_a
      // with this target's own operator, G alpha = V_a^T b, x0 = V_a alpha
      const int sl = d.slot + parity_base;
      const SlotMeta mt = p.slotMeta[sl];
      const int a = mt.a;
      if (mt.timestep == tstep && mt.N == N && a > 0 && a * a <= (m + 1) * m) {
        const double* V = p.slotV + (size_t)sl * (p.max_a + 1) * p.slot_ld;
        double* G = sm.Hr;                       // a x a, column-major
        for (int k = 0; k < a; ++k) {
          const double* vk = V + (size_t)k * p.slot_ld;
          double av[EPT];
#pragma unroll
          for (int e = 0; e < EPT; ++e) {
            const int pp = tid + e * NT;
            av[e] = 0.0;
            if (pp < N) {
              const int pe = min(pp + H, N - 1), pw = max(pp - H, 0);
              const int pn = min(pp + 1, N - 1), ps = max(pp - 1, 0);
              double t = cd * vk[pp];
              t = fma(cE[e], vk[pe], t);
              t = fma(cW[e], vk[pw], t);
              t = fma(cN[e], vk[pn], t);
              av[e] = fma(cS[e], vk[ps], t);
            }
          }
          block_partials<NT>(a, [&](int l) {
            const double* vl = V + (size_t)l * p.slot_ld;
            double s = 0.0;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
              const int pp = tid + e * NT;
              if (pp < N) s = fma(vl[pp], av[e], s);
            }
            return s;
          }, sm.red);
          if (warp == 0)
            for (int l = lane; l < a; l += 32) G[l + k * a] = cross_warp<NT>(sm.red, l);
          __syncthreads();                       // partials of the next column reuse red
        }
        double bv[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) bv[e] = bval(tid + e * NT);
        block_partials<NT>(a, [&](int l) {
          const double* vl = V + (size_t)l * p.slot_ld;
          double s = 0.0;
#pragma unroll
          for (int e = 0; e < EPT; ++e) {
            const int pp = tid + e * NT;
            if (pp < N) s = fma(vl[pp], bv[e], s);
          }
          return s;
        }, sm.red);
        if (warp == 0) {
          for (int l = lane; l < a; l += 32) sm.hb[l] = cross_warp<NT>(sm.red, l);
          __syncwarp();
          const bool ok = lu_solve_warp(G, a, sm.hb, lane);
          if (lane == 0) sm.fl[5] = ok;
        }
        __syncthreads();
        if (sm.fl[5]) {
#pragma unroll
          for (int e = 0; e < EPT; ++e) {
            const int pp = tid + e * NT;
            if (pp < N) {
              double xv = 0.0;
              for (int i = 0; i < a; ++i) xv = fma(sm.hb[i], V[(size_t)i * p.slot_ld + pp], xv);
              sm.xs[pp] = xv;
            }
          }
        }
        proj_flops = (unsigned long long)(a * (9 + 2 * a) + 4 * a) * (unsigned long long)N;
      }
    }
    __syncthreads();
    double w[EPT];
    auto residual = [&]() { residual_of(sm.xs, w); };
    int steps = 0, status = KP_NOT_CONVERGED, cycle = 0;
    double bnorm = 0.0, beta = 0.0;
    unsigned long long bicg_fl = 0;            // flops per unknown of a BiCGSTAB seed solve
    const bool bicg = BICG && capture;
    if (BICG && bicg) {
      // Sec. 3, Phase 1 as printed: BiCGSTAB (van der Vorst 1992) on the seed,
      // restarted from the true residual when the updated one has drifted.
      // The key vectors of the first sweep (r_0, then s_k and r_k of every
      // iteration), orthonormalised by CGS2 against the ones kept before, are
      // the stored basis V_a; A_proj = V_a^T A V_a is formed explicitly for
      // the targets (BiCGSTAB has no Hessenberg relation).
      double* rh = slot(0);                    // shadow residual
      double* rv = slot(1);                    // r
      double* pv = slot(2);                    // search direction p
      double* vv = slot(3);                    // A p
      double* sv = slot(4);                    // intermediate residual s
      // block sums of nv values fn(i) into sm.hb[0..nv)
      auto reduce = [&](int nv, auto&& fn) {
        block_partials<NT>(nv, fn, sm.red);
        if (warp == 0)
          for (int i = lane; i < nv; i += 32) sm.hb[i] = cross_warp<NT>(sm.red, i);
        __syncthreads();
      };
      auto apply_full = [&](const double* v) {   // w = A v
        apply_off(v, w);
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          w[k] = pp < N ? fma(cd, v[pp], w[k]) : 0.0;
        }
      };
      int nkeep = 0;
      // keep u (this thread's points) as basis vector nkeep if it adds a direction
      auto keep = [&](const double* u) {
        if (nkeep >= p.cap_a) return;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          w[k] = pp < N ? u[pp] : 0.0;
        }
        double n0 = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
          reduce(nkeep + 1, [&](int i) {
            double s = 0.0;
            if (i < nkeep) {
              const double* vi = capV + (size_t)i * p.cap_ld;
#pragma unroll
              for (int k = 0; k < EPT; ++k) {
                const int pp = tid + k * NT;
                if (pp < N) s = fma(vi[pp], w[k], s);
              }
            } else {
#pragma unroll
              for (int k = 0; k < EPT; ++k) s = fma(w[k], w[k], s);
            }
            return s;
          });
          if (pass == 0) n0 = sm.hb[nkeep];
          for (int i = 0; i < nkeep; ++i) {
            const double hi = sm.hb[i];
            const double* vi = capV + (size_t)i * p.cap_ld;
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
              const int pp = tid + k * NT;
              if (pp < N) w[k] = fma(-hi, vi[pp], w[k]);
            }
          }
        }
        reduce(1, [&](int) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < EPT; ++k) s = fma(w[k], w[k], s);
          return s;
        });
        const double n1 = sm.hb[0];
        bicg_fl += 8ull * nkeep + 7ull;
        if (!(n1 > 1e-20 * n0)) return;        // no new direction (norm ratio 1e-10)
        const double inv = 1.0 / sqrt(n1);
        double* vn = capV + (size_t)nkeep * p.cap_ld;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          if (pp < N) vn[pp] = w[k] * inv;
        }
        ++nkeep;
      };
      int sweep = 0;
      for (;;) {
        // true residual r = b - A x (x = 0 for the first sweep of a seed)
        if (sweep == 0 && p.x0_mode == X0_ZERO) {
#pragma unroll
          for (int k = 0; k < EPT; ++k) w[k] = bval(tid + k * NT);
        } else {
          __syncthreads();
          residual();
        }
        reduce(2, [&](int i) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const double bv = bval(tid + k * NT);
            s += (i == 0) ? bv * bv : w[k] * w[k];
          }
          return s;
        });
        bnorm = sqrt(sm.hb[0]);
        beta = sqrt(sm.hb[1]);
        bicg_fl += 12;
        if (beta <= p.tol * bnorm) { status = KP_OK; break; }
        if (!isfinite(beta)) { status = KP_BREAKDOWN; break; }
        if (steps >= p.maxit) break;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          rh[pp] = w[k];
          rv[pp] = w[k];
          pv[pp] = 0.0;
          vv[pp] = 0.0;
        }
        const bool keeping = sweep == 0;
        if (keeping) keep(rv);
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        const int steps0 = steps;
        while (steps < p.maxit) {
          reduce(1, [&](int) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fma(rh[tid + k * NT], rv[tid + k * NT], s);
            return s;
          });
          const double rho = sm.hb[0];
          if (rho == 0.0) break;
          const double bt = (rho / rho_old) * (alpha / omega);
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            pv[pp] = fma(bt, fma(-omega, vv[pp], pv[pp]), rv[pp]);
          }
          __syncthreads();                     // p complete for the stencil
          apply_full(pv);
          reduce(1, [&](int) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fma(rh[tid + k * NT], w[k], s);
            return s;
          });
          alpha = rho / sm.hb[0];
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            vv[pp] = w[k];
            sv[pp] = fma(-alpha, w[k], rv[pp]);
          }
          ++steps;
          bicg_fl += 42;
          reduce(1, [&](int) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fma(sv[tid + k * NT], sv[tid + k * NT], s);
            return s;
          });
          if (sqrt(sm.hb[0]) <= p.tol * bnorm) {
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
              const int pp = tid + k * NT;
              sm.xs[pp] = fma(alpha, pv[pp], sm.xs[pp]);
            }
            if (keeping) keep(sv);
            break;
          }
          __syncthreads();                     // s complete for the stencil
          apply_full(sv);                      // t = A s
          reduce(2, [&](int i) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fma(w[k], i == 0 ? sv[tid + k * NT] : w[k], s);
            return s;
          });
          omega = sm.hb[1] > 0.0 ? sm.hb[0] / sm.hb[1] : 0.0;
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            sm.xs[pp] = fma(omega, sv[pp], fma(alpha, pv[pp], sm.xs[pp]));
            rv[pp] = fma(-omega, w[k], sv[pp]);
          }
          if (keeping) { keep(sv); keep(rv); }
          reduce(1, [&](int) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fma(rv[tid + k * NT], rv[tid + k * NT], s);
            return s;
          });
          if (sqrt(sm.hb[0]) <= p.tol * bnorm || omega == 0.0) break;
          rho_old = rho;
        }
        if (steps == steps0) { status = KP_BREAKDOWN; break; }   // a sweep without progress
        ++sweep;
      }
      // A_proj = V_a^T A V_a, column by column, into the seed's slot
      const int a = nkeep;
      const int sl = cidx;
      double* R = p.slotR + (size_t)sl * (p.max_a + 1) * p.max_a;
      __syncthreads();                         // kept vectors complete for the stencil
      for (int kc = 0; kc < a; ++kc) {
        apply_full(capV + (size_t)kc * p.cap_ld);
        reduce(a, [&](int l) {
          const double* vl = capV + (size_t)l * p.cap_ld;
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            if (pp < N) s = fma(vl[pp], w[k], s);
          }
          return s;
        });
        for (int l = tid; l < a; l += NT) R[l + (size_t)kc * (p.max_a + 1)] = sm.hb[l];
      }
      bicg_fl += (unsigned long long)a * (9 + 2 * a);
      if (tid == 0) {
        SlotMeta mt;
        mt.a = a;
        mt.has_next = 0;
        mt.timestep = tstep;
        mt.N = N;
        mt.lsq = 0;
        mt.nrot = 0;
        mt.dense = 1;
        mt.pad_ = 0;
        p.slotMeta[sl] = mt;
      }
      __syncthreads();
    }
    const int npic = bicg ? 0 : (PICARD && p.picard > 1) ? p.picard : 1;

    for (int pk = 0; pk < npic; ++pk) {
      if (PICARD && pk > 0) {
        // Picard iteration k = pk + 1 (Sec. 2.3): the nonlinear term lagged on
        // the latest iterate m^{n,(k-1)} (in shared memory), the same right-hand
        // side, GMRES warm-started from that iterate
        __syncthreads();
        set_coeffs(sm.xs, false);
        status = KP_NOT_CONVERGED;
        capture = false;                         // the stored basis is the first solve's
      }
      if (pk == 0 && p.x0_mode == X0_ZERO) {     // r = b, no operator application needed
#pragma unroll
        for (int k = 0; k < EPT; ++k) w[k] = bval(tid + k * NT);
      } else {
        residual();
      }
      block_partials<NT>(2, [&](int i) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          const double bv = pp < N ? d.b[pp] : 0.0;
          s += (i == 0) ? bv * bv : w[k] * w[k];
        }
        return s;
      }, sm.red);
      if (tid == 0) {
        sm.sc[0] = sqrt(cross_warp<NT>(sm.red, 0));
        sm.sc[1] = sqrt(cross_warp<NT>(sm.red, 1));
      }
      __syncthreads();
      bnorm = sm.sc[0];
      beta = sm.sc[1];

      if (bnorm == 0.0) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) sm.xs[tid + k * NT] = 0.0;
        beta = 0.0;
        status = KP_OK;
      }
      while (status == KP_NOT_CONVERGED) {
        if (beta <= p.tol * bnorm) { status = KP_OK; break; }
        if (!isfinite(beta)) { status = KP_BREAKDOWN; break; }
        if (steps >= p.maxit) break;
        {
          const double ib = 1.0 / beta;
          double* v0 = slot(0);
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            v0[pp] = w[k] * ib;
            if (capture && cycle == 0 && pp < N) capV[pp] = w[k] * ib;
          }
          if (tid == 0) sm.g[0] = beta;
        }
        int kdone = 0;
        int brk = 0;
        // Givens update of Hessenberg column j once h_{j+1,j}^2 = hn2 is known
        // (one lane): rotations, residual estimate, convergence flags.
        auto givens_step = [&](int j, double hn2) {
          const double ihn = hn2 > 0.0 ? rsqrt(hn2) : 0.0;
          const double hn = hn2 * ihn;
          const int b = !(hn2 > 1e-28 * sm.sc[2]);  // h_{j+1,j} <= 1e-14 ||A v_j||
          sm.Hr[j + j * ld] += cd;                 // H_A = H_{A - cd I} + cd I
          sm.Hr[(j + 1) + j * ld] = hn;
          if (capture && cycle == 0 && j < p.cap_a) {
            for (int i = 0; i <= j + 1; ++i) capH[i + j * (p.cap_a + 1)] = sm.Hr[i + j * ld];
          }
          for (int i = 0; i < j; ++i) {
            const double t1 = sm.Hr[i + j * ld], t2 = sm.Hr[(i + 1) + j * ld];
            sm.Hr[i + j * ld] = sm.cs[i] * t1 + sm.sn[i] * t2;
            sm.Hr[(i + 1) + j * ld] = -sm.sn[i] * t1 + sm.cs[i] * t2;
          }
          const double a0 = sm.Hr[j + j * ld];
          const double rr = a0 * a0 + hn2;
          const double ir = rsqrt(rr);
          const double c = a0 * ir, s = hn * ir;
          sm.cs[j] = c;
          sm.sn[j] = s;
          sm.Hr[j + j * ld] = rr * ir;
          sm.rinv[j] = ir;
          sm.Hr[(j + 1) + j * ld] = 0.0;
          sm.g[j + 1] = -s * sm.g[j];
          sm.g[j] = c * sm.g[j];
          const double res = fabs(sm.g[j + 1]);
          sm.sc[3] = ihn;
          sm.fl[1] = b;
          // fixed basis dimension: the capture cycle reaches cap_a steps
          // before the residual test may end it
          const bool short_of_a = p.fixed_a && capture && cycle == 0 && j + 1 < p.cap_a;
          sm.fl[2] = (res <= p.tol * bnorm && !short_of_a) || b || (steps >= p.maxit) || (j + 1 == m);
        };
        for (int j = 0; j < m; ++j) {
          __syncthreads();                       // v_j complete
          apply_off(slot(j), w);
          ++steps;
          const int nh = j + 1;
          auto dots = [&](int i) {
            double s = 0.0;
            if (i < nh) {
              const double* vi = slot(i);
#pragma unroll
              for (int k = 0; k < EPT; ++k) s += vi[tid + k * NT] * w[k];
            } else {
#pragma unroll
              for (int k = 0; k < EPT; ++k) s += w[k] * w[k];
            }
            return s;
          };
          // CGS pass 1: h_i = <v_i, w> and ||w||^2 in one batched reduction
          block_partials<NT>(nh + 1, dots, sm.red);
          if (warp == 0) {
            double sq = 0.0;
            for (int i = lane; i <= nh; i += 32) {
              const double s = cross_warp<NT>(sm.red, i);
              sm.hb[i] = s;
              if (i < nh) { sm.Hr[i + j * ld] = s; sq += s * s; }
            }
            sq = warp_sum(sq);
            if (lane == 0) {
              const double ww0 = sm.hb[nh];
              sm.sc[2] = ww0;
              // ||w_1||^2 = ||w||^2 - ||h||^2, accurate to a few ulps of ||w||^2
              // while at most half of it is removed; otherwise the second pass
              // measures ||w_1||^2 in its reduction
              const int big = ww0 - sq < 0.5 * ww0;
              sm.fl[4] = big;
              sm.sc[4] = ww0 - sq;
              // second pass always (CGS2), or only when the first removed over
              // half of ||w||^2 (DGKS)
              const int pass2 = (p.reorth == 0) || big;
              sm.fl[0] = pass2;
              if (!pass2) givens_step(j, ww0 - sq);
            }
          }
          __syncthreads();
          for (int i = 0; i < nh; ++i) {
            const double hi = sm.hb[i];
            const double* vi = slot(i);
#pragma unroll
            for (int k = 0; k < EPT; ++k) w[k] = fma(-hi, vi[tid + k * NT], w[k]);
          }
          if (sm.fl[0]) {
            // CGS pass 2 (reorthogonalisation), with ||w_1||^2 in the same
            // reduction when pass 1 removed most of ||w||^2;
            // ||w_2||^2 = ||w_1||^2 - ||h_2||^2 (h_2 = O(eps) after pass 1), checked
            const int big = sm.fl[4];
            block_partials<NT>(big ? nh + 1 : nh, dots, sm.red);
            if (warp == 0) {
              double sq = 0.0;
              for (int i = lane; i < (big ? nh + 1 : nh); i += 32) {
                const double s = cross_warp<NT>(sm.red, i);
                sm.hb[i] = s;
                if (i < nh) { sm.Hr[i + j * ld] += s; sq += s * s; }
              }
              sq = warp_sum(sq);
              if (lane == 0) {
                const double ww1 = big ? sm.hb[nh] : sm.sc[4];
                const int exact = sq > 0.25 * ww1;     // large correction: recompute the norm
                sm.fl[3] = exact;
                if (!exact) givens_step(j, ww1 - sq);
              }
            }
            __syncthreads();
            for (int i = 0; i < nh; ++i) {
              const double hi = sm.hb[i];
              const double* vi = slot(i);
#pragma unroll
              for (int k = 0; k < EPT; ++k) w[k] = fma(-hi, vi[tid + k * NT], w[k]);
            }
            if (sm.fl[3]) {
              block_partials<NT>(1, [&](int) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < EPT; ++k) s += w[k] * w[k];
                return s;
              }, sm.red);
              if (tid == 0) givens_step(j, cross_warp<NT>(sm.red, 0));
              __syncthreads();
            }
          }
          brk = sm.fl[1];
          kdone = j + 1;
          if (!brk) {
            const double ih = sm.sc[3];
            double* vn = slot(j + 1);
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
              const int pp = tid + k * NT;
              vn[pp] = w[k] * ih;
              if (capture && cycle == 0 && j + 1 <= p.cap_a && pp < N)
                capV[(size_t)(j + 1) * p.cap_ld + pp] = w[k] * ih;
            }
          }
          if (sm.fl[2]) break;
        }
        // y = R^{-1} g: column-oriented back substitution on warp 0 (lane l owns
        // rows l and l+32), reciprocal pivots stored by the Givens step
        if (warp == 0) {
          double g0 = (lane < kdone) ? sm.g[lane] : 0.0;
          double g1 = (lane + 32 < kdone) ? sm.g[lane + 32] : 0.0;
          for (int i = kdone - 1; i >= 0; --i) {
            const double gi = __shfl_sync(kFull, i < 32 ? g0 : g1, i & 31);
            const double yi = gi * sm.rinv[i];
            if (lane == 0) sm.y[i] = yi;
            if (lane < i) g0 = fma(-sm.Hr[lane + i * ld], yi, g0);
            if (lane + 32 < i) g1 = fma(-sm.Hr[(lane + 32) + i * ld], yi, g1);
          }
        }
        if (tid == 0) {
          if (capture && cycle == 0) {
            const int a = kdone < p.cap_a ? kdone : p.cap_a;
            const int hn = (a < kdone) || !brk;
            if (p.factor) {
              // fused basis store: factor H_a of the slot just written
              SlotMeta mt;
              const int sl = cidx;
              double* rot = p.slotRot + (size_t)sl * 3 * p.max_a;
              factor_hessenberg(capH, p.cap_a + 1, a, hn,
                                p.slotR + (size_t)sl * (p.max_a + 1) * p.max_a, rot,
                                rot + 2 * p.max_a, &mt.lsq, &mt.nrot);
              mt.a = a;
              mt.has_next = hn;
              mt.timestep = tstep;
              mt.N = N;
              mt.dense = mt.pad_ = 0;
              p.slotMeta[sl] = mt;
            } else {
              p.capMeta[sysi].a = a;
              p.capMeta[sysi].has_next = hn;
              p.capMeta[sysi].N = N;
              p.capMeta[sysi].valid = 1;
            }
          }
        }
        __syncthreads();
        for (int i = 0; i < kdone; ++i) {
          const double yi = sm.y[i];
          const double* vi = slot(i);
#pragma unroll
          for (int k = 0; k < EPT; ++k) sm.xs[tid + k * NT] = fma(yi, vi[tid + k * NT], sm.xs[tid + k * NT]);
        }
        __syncthreads();
        residual();                              // true FP64 residual
        block_partials<NT>(1, [&](int) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < EPT; ++k) s += w[k] * w[k];
          return s;
        }, sm.red);
        if (tid == 0) sm.sc[1] = sqrt(cross_warp<NT>(sm.red, 0));
        __syncthreads();
        beta = sm.sc[1];
        ++cycle;
      }
      if (pk == 0 && capture && cycle == 0 && tid == 0) {   // converged before any step: empty basis
        if (p.factor) {
          SlotMeta mt;
          mt.a = 0;
          mt.has_next = 0;
          mt.timestep = tstep;
          mt.N = N;
          mt.lsq = 0;
          mt.nrot = 0;
          mt.dense = mt.pad_ = 0;
          p.slotMeta[cidx] = mt;
        } else {
          p.capMeta[sysi].a = 0;
          p.capMeta[sysi].has_next = 0;
          p.capMeta[sysi].N = N;
          p.capMeta[sysi].valid = 1;
        }
      }
    }                                          // Picard iterations
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      if (pp < N) d.x[pp] = sm.xs[pp];
    }
    if (SCORE && score_on && tstep == *p.step_end - 1) {
      // last timestep of the run: the score of its own solution m^n (the
      // next run's first item writes the same values again from its input)
      double* sc = d.score + (size_t)tstep * p.score_stride;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        if (pp < N) {
          const int i = pp / H, j = pp - i * H;
          const double xe = i + 1 < W ? sm.xs[pp + H] : 0.0, xw = i > 0 ? sm.xs[pp - H] : 0.0;
          const double xn = j + 1 < H ? sm.xs[pp + 1] : 0.0, xs_ = j > 0 ? sm.xs[pp - 1] : 0.0;
          sc[pp] = (xe - xw) * s_i2h;
          sc[N + pp] = (xn - xs_) * s_i2h;
        }
      }
    }
    if (tid == 0) {
      const double rel = bnorm > 0.0 ? beta / bnorm : 0.0;
      if (p.info) {
        kp_info inf;
        inf.iters = steps;
        inf.status = status;
        inf.rel_res = rel;
        p.info[sysi] = inf;
      }
      if (p.acc) {
        StepAcc* a = p.acc + tstep;
        const unsigned long long fl = (bicg ? bicg_fl : gmres_flops(steps, m)) * (unsigned long long)N;
        if (p.acc_kind == 0) {
          atomicAdd(&a->seed_iters, (unsigned long long)steps);
          atomicAdd(&a->seed_flops, fl);
        } else {
          atomicAdd(&a->tgt_iters, (unsigned long long)steps);
          atomicAdd(&a->tgt_flops, fl);
          atomicMax(&a->tgt_max_iters, (unsigned int)steps);
          atomicMax(&a->max_res_bits, (unsigned long long)__double_as_longlong(rel));
          if (proj_flops) atomicAdd(&a->proj_flops, proj_flops);
        }
        if (status != KP_OK) atomicAdd(&a->not_converged, 1u);
      }
    }
    if (p.done) {                              // release m^n of this system
      __threadfence();
      __syncthreads();
      if (tid == 0) st_release_gpu(p.done + sysi, tstep + 1 - *p.run_start);
    }
    __syncthreads();                           // shared memory reused by the next item
    if (!p.queue && ++kstep == nstep) { kstep = 0; sysi += gridDim.x; }
  }
  if (p.pdl & 2) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Raise the kernel's dynamic shared-memory limit to the device maximum, so
// that launches with different windows (seeds, targets) never lower it.
template <typename K>
static cudaError_t allow_max_smem(K k, size_t smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <int EPT, int NT, int MINB, int VAR>
static cudaError_t launch_one(const GmresParams& p, size_t smem, cudaStream_t st) {
  auto k = gmres_fp64_kernel<EPT, NT, MINB, VAR>;
  cudaError_t e = allow_max_smem(k, smem);
  if (e != cudaSuccess) return e;
  const int grid = p.grid > 0 ? p.grid : p.nsys;
  if (p.pdl & 2) {
    // programmatic dependent launch: the blocks may start while the previous
    // kernel of the stream still runs (it signals at entry)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, p);
  }
  k<<<grid, NT, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace
}  // namespace kp
