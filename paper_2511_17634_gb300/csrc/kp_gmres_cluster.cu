// kp_gmres_cluster.cu -- the mixed-precision solver of kp_gmres_mixed.cu for
// grids too large for one SM (128x128 = 16384 unknowns): a thread-block
// cluster of CS CTAs per system, CTA r holding columns [r*W/CS, (r+1)*W/CS)
// of every vector (whole columns, so north/south neighbours stay local).
//
//  * East/west neighbours across a slice edge are read from the adjacent
//    CTA's shared memory (distributed shared memory), or from its slice of
//    the device workspace for Krylov vectors beyond the shared-memory window.
//  * Inner products: FP32 per thread and warp, FP64 across warps, then the CS
//    per-CTA partials are summed in rank order by every CTA (one cluster
//    barrier, double-buffered partials), so all CTAs hold bit-identical
//    coefficients and run the FP64 Hessenberg / Givens updates redundantly
//    instead of broadcasting them.
//  * Same stopping rules as the one-block mixed kernel: FP32 Krylov inside
//    iterative refinement on the true residual.  The refinement's
//    high-precision arithmetic -- x, the operator coefficients, b - A x --
//    is double-float (kp_dd.cuh, about 48 bits) on the FP32 pipe instead of
//    FP64: on GB300 the FP64 pipe issues 2 operations per clock per SM and
//    the FP64 residuals, judge and coefficient set-up held it busy over half
//    of the kernel.  The residual's error is a few units of 2^-44 times
//    ||b||, far under every tolerance the solver is asked for (>= 1e-12).
#include <cooperative_groups.h>

#include "kp_dd.cuh"
#include "kp_internal.cuh"

namespace cg = cooperative_groups;

namespace kp {
namespace {

// MINB resident CTAs per SM: 2 (the default) lets two systems' clusters
// share the SMs, so one system's barriers and serial FP64 work overlap the
// other's vector work (registers capped at 128, a smaller shared-memory
// window); 1 gives one CTA the whole SM.
template <int EPT, int NT, int CS, int MINB>
__global__ void __launch_bounds__(NT, MINB) gmres_cluster_kernel(const GmresParams p) {
  constexpr int NWARPS = NT / 32;
  extern __shared__ __align__(16) double smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int npad = EPT * NT;
  const int m = p.m;
  const int ld = m + 1;
  // shared-memory carve (identical offsets in every CTA of the cluster)
  float* xh = reinterpret_cast<float*>(smem_raw);  // [npad] slice of x, double-float hi
  float* xl = xh + npad;                           // [npad] and lo parts
  double* red = smem_raw + npad;                  // [NWARPS][kMaxV]
  float* red32 = reinterpret_cast<float*>(red);    // FP32 per-warp partials (same space)
  double* hb = red + NWARPS * kMaxV;              // [kMaxV] cluster sums
  double* cpart = hb + kMaxV;                     // [2][kMaxV] per-CTA partials
  double* Hr = cpart + 2 * kMaxV;                 // [(m+1) m]
  double* gv = Hr + (m + 1) * m;
  double* cs = gv + (m + 1);
  double* sn = cs + m;
  double* yv = sn + m;
  double* rinv = yv + m;
  double* sc = rinv + m;                          // [8]
  int* fl = reinterpret_cast<int*>(sc + 8);       // [8]
  float* hbf = reinterpret_cast<float*>(fl + 8);  // [kMaxV] the cluster sums in FP32
  float* V = hbf + kMaxV;                         // [S][npad]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sysi = blockIdx.x / CS;
  const int cta0 = blockIdx.x - rank;             // first CTA of this cluster
  const size_t spill_per = (size_t)(m + 1 - p.S) * npad;
  auto vloc = [&](int i) -> float* {
    return i < p.S ? V + (size_t)i * npad : p.spill32 + (size_t)blockIdx.x * spill_per + (size_t)(i - p.S) * npad;
  };
  auto vrem = [&](int i, int r) -> const float* {
    return i < p.S ? cluster.map_shared_rank(V + (size_t)i * npad, r)
                   : p.spill32 + (size_t)(cta0 + r) * spill_per + (size_t)(i - p.S) * npad;
  };
  int tstep = 0;
  if (p.step) {
    tstep = *p.step + p.step_offset;
    if (tstep >= *p.step_end) return;            // uniform over the whole grid
  }
  if (sysi >= p.nsys) return;                     // uniform over the cluster
  const int parity_base = slot_set_base(p, tstep);
  const double bsc = p.b_scale;
  const double kEta = p.inner_eta > 0.0 ? p.inner_eta : 1e-5;

  const SysDesc d = p.sys[sysi];
  const int H = d.H, W = d.W, N = H * W;
  const int SL = N / CS;                          // slice length (whole columns)
  const int base = rank * SL;
  const double hh = d.h;
  const double g2 = p.step ? p.g2_sched[tstep] : d.g2;
  // solved as (A / s) x = b / s with s = b_scale: the scale goes on the
  // operator constants once per solve instead of on every point of b
  const double osc = bsc != 0.0 ? 1.0 / bsc : 1.0;
  const double cc = g2 / (2.0 * hh * hh) * osc;
  const double ee = g2 / (8.0 * hh * hh) * osc;
  const double cd = (1.0 / d.dt + 2.0 * g2 / (hh * hh)) * osc;
  const double i2h = osc / (2.0 * hh);
  const float ccf = (float)cc;
  const bool capture = p.capV32 != nullptr;
  const int cidx = p.factor ? parity_base + sysi : sysi;
  float* capV = capture ? p.capV32 + (size_t)cidx * (p.cap_a + 1) * p.cap_ld : nullptr;
  double* capH = capture ? p.capH + (size_t)cidx * (p.cap_a + 1) * p.cap_a : nullptr;

  // FP32 q_x, q_y for the Krylov operator; double-float E and N coefficients
  // cE = q_x - c, cN = q_y - c for the residual (cW = -2c - cE, cS = -2c - cN),
  // from the FP64 field split without FP64 instructions.  In the judge mode
  // (a given guess) the warm start's residual norm comes out of the same
  // loads: sw = sum of r_warm^2 over this thread's points.
  const bool judge = p.x0_mode == X0_GUESS_PROJECT;
  const dd ccd = dd_from_double(cc), eed = dd_from_double(ee), cdd = dd_from_double(cd), i2hd = dd_from_double(i2h);
  const dd c2d = dd_from_double(2.0 * cc);
  dd cE[EPT], cN[EPT];
  float qxf[EPT], qyf[EPT];
  unsigned msk = 0;                               // 4 neighbour bits per point
  float sw = 0.f;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int l = tid + k * NT, pp = base + l;
    dd qx = {0.f, 0.f}, qy = {0.f, 0.f};
    if (l < SL) {
      const int i = pp / H, j = pp - i * H;
      const unsigned mk = (i + 1 < W ? 1u : 0u) | (i > 0 ? 2u : 0u) | (j + 1 < H ? 4u : 0u) | (j > 0 ? 8u : 0u);
      msk |= mk << (4 * k);
      const dd mE = dd_from_double((mk & 1u) ? d.mt[pp + H] : 0.0);
      const dd mW = dd_from_double((mk & 2u) ? d.mt[pp - H] : 0.0);
      const dd mN = dd_from_double((mk & 4u) ? d.mt[pp + 1] : 0.0);
      const dd mS = dd_from_double((mk & 8u) ? d.mt[pp - 1] : 0.0);
      qx = dd_mul(eed, dd_sub(mW, mE));
      qy = dd_mul(eed, dd_sub(mS, mN));
      if (d.fx) qx = dd_add(qx, dd_mul(dd_from_double(d.fx[pp]), i2hd));
      if (d.fy) qy = dd_add(qy, dd_mul(dd_from_double(d.fy[pp]), i2hd));
      cE[k] = dd_sub(qx, ccd);
      cN[k] = dd_sub(qy, ccd);
      if (judge) {
        const dd mC = dd_from_double(d.mt[pp]);
        dd t = dd_sub(dd_from_double(d.b[pp]), dd_mul(cdd, mC));
        t = dd_sub(t, dd_mul(cE[k], dd_sub(mE, mW)));
        t = dd_sub(t, dd_mul(cN[k], dd_sub(mN, mS)));
        t = dd_add(t, dd_mul(c2d, dd_add(mW, mS)));
        sw = fmaf(t.hi, t.hi, sw);
      }
    } else {
      cE[k] = cN[k] = dd{0.f, 0.f};
    }
    qxf[k] = qx.hi;
    qyf[k] = qy.hi;
  }
  auto mbits = [&](int k) { return (msk >> (4 * k)) & 15u; };
  const float* xh_next = rank + 1 < CS ? cluster.map_shared_rank(xh, rank + 1) : nullptr;
  const float* xh_prev = rank > 0 ? cluster.map_shared_rank(xh, rank - 1) : nullptr;
  const float* xl_next = rank + 1 < CS ? cluster.map_shared_rank(xl, rank + 1) : nullptr;
  const float* xl_prev = rank > 0 ? cluster.map_shared_rank(xl, rank - 1) : nullptr;
  // r = b - A x in double-float (A x = cd x + cE (xE - xW) - 2c xW + cN (xN -
  // xS) - 2c xS); out = its hi part, which is all the FP32 Krylov and the
  // norms need
  auto residual_of = [&](float (&out)[EPT]) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int l = tid + k * NT;
      out[k] = 0.f;
      if (l < SL) {
        const unsigned mk = mbits(k);
        const dd z = {0.f, 0.f};
        const dd xE = (mk & 1u) ? (l + H < SL ? dd{xh[l + H], xl[l + H]} : dd{xh_next[l + H - SL], xl_next[l + H - SL]}) : z;
        const dd xW = (mk & 2u) ? (l - H >= 0 ? dd{xh[l - H], xl[l - H]} : dd{xh_prev[l - H + SL], xl_prev[l - H + SL]}) : z;
        const dd xN = (mk & 4u) ? dd{xh[l + 1], xl[l + 1]} : z;
        const dd xS = (mk & 8u) ? dd{xh[l - 1], xl[l - 1]} : z;
        dd t = dd_sub(dd_from_double(d.b[base + l]), dd_mul(cdd, dd{xh[l], xl[l]}));
        t = dd_sub(t, dd_mul(cE[k], dd_sub(xE, xW)));
        t = dd_sub(t, dd_mul(cN[k], dd_sub(xN, xS)));
        t = dd_add(t, dd_mul(c2d, dd_add(xW, xS)));
        out[k] = t.hi;
      }
    }
  };
  auto apply32 = [&](int vi, float (&out)[EPT]) {
    const float* v = vloc(vi);
    const float* vn = rank + 1 < CS ? vrem(vi, rank + 1) : nullptr;
    const float* vp = rank > 0 ? vrem(vi, rank - 1) : nullptr;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int l = tid + k * NT;
      out[k] = 0.f;
      if (l < SL) {
        const unsigned mk = mbits(k);
        const float xE = (mk & 1u) ? (l + H < SL ? v[l + H] : vn[l + H - SL]) : 0.f;
        const float xW = (mk & 2u) ? (l - H >= 0 ? v[l - H] : vp[l - H + SL]) : 0.f;
        const float xN = (mk & 4u) ? v[l + 1] : 0.f;
        const float xS = (mk & 8u) ? v[l - 1] : 0.f;
        out[k] = -ccf * (xE + xW + xN + xS) + qxf[k] * (xE - xW) + qyf[k] * (xN - xS);
      }
    }
  };
  auto bhi = [&](int l) { return (l < SL) ? dd_from_double(d.b[base + l]).hi : 0.f; };
  int buf = 0;
  // cluster-wide sums of nv values whose per-warp partials are in red;
  // result in hb[0..nv) of every CTA (identical: the same pairwise sum of the
  // CS partials in every CTA).  f32: the partials are FP32, summed across
  // warps on the FP32 pipe.  tail(): warp 0's work on the sums (Hessenberg
  // column, Givens step), run before the CTA barrier that publishes them.
  auto cluster_sum = [&](int nv, bool f32, auto&& tail) {
    if (warp == 0) {
      if (f32) cross_warp_f32<NT>(red32, nv, cpart + buf * kMaxV, lane);
      else
        for (int i = lane; i < nv; i += 32) cpart[buf * kMaxV + i] = cross_warp<NT>(red, i);
    }
    cluster.sync();
    if (warp == 0) {
      for (int i = lane; i < nv; i += 32) {
        double v[CS];
#pragma unroll
        for (int r = 0; r < CS; ++r) v[r] = cluster.map_shared_rank(cpart + buf * kMaxV, r)[i];
#pragma unroll
        for (int w = 1; w < CS; w *= 2)
#pragma unroll
          for (int r = 0; r + w < CS; r += 2 * w) v[r] += v[r + w];
        hb[i] = v[0];
        hbf[i] = (float)v[0];                     // converted once for the vector updates
      }
      __syncwarp();
      tail();
    }
    __syncthreads();
    buf ^= 1;
  };
  auto no_tail = [] {};

  // initial guess, split into double-float without FP64 instructions
  auto load_x = [&](const double* src) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int l = tid + k * NT;
      const dd v = (src && l < SL) ? dd_from_double(src[base + l]) : dd{0.f, 0.f};
      xh[l] = v.hi;
      xl[l] = v.lo;
    }
  };
  if (p.gdelta && (p.x0_mode == X0_READ || judge)) {
    // the learned guess x_init = m~ + dt rho net, from the network's FP32
    // output, in double-float
    const float s = (float)(p.grho[sysi] / p.gdiv);
    const float* dl = p.gdelta + (size_t)sysi * p.gdelta_ld + base;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int l = tid + k * NT;
      const dd v = l < SL ? dd_add_f(dd_from_double(d.mt[base + l]), s * dl[l]) : dd{0.f, 0.f};
      xh[l] = v.hi;
      xl[l] = v.lo;
    }
  } else {
    load_x(p.x0_mode == X0_READ || judge ? d.x : p.x0_mode == X0_WARM ? d.mt : nullptr);
  }
  unsigned long long proj_flops = 0;
  float r[EPT];
  auto residual = [&]() { residual_of(r); };
  bool r_current = false;                         // r already holds b - A x0
  if (judge) {
    // the judge of a given guess (as in the one-block mixed solver): the
    // guess's true residual against the warm start's (sw, from the set-up);
    // a kept guess is projected, the warm start starts as is
    cluster.sync();                               // x_init slices visible cluster-wide
    residual();
    block_partials_f32x<NT>(2, [&](int i) {
      float s = 0.f;
      if (i == 0) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) s = fmaf(r[k], r[k], s);
      } else {
        s = sw;
      }
      return s;
    }, red32);
    cluster_sum(2, true, no_tail);               // (its barrier also ends every read of x_init)
    const bool warm_won = hb[1] < hb[0];          // the same in every CTA
    if (warm_won) load_x(d.mt);
    r_current = !warm_won;
    proj_flops = 26ull * (unsigned long long)N;
    // Sec. 3, Phase 2 on the residual of the guess: c = V^T r,
    // alpha = H_a^{-1} c, x0 = x_init + V alpha, the sums cluster-wide
    const int sl = d.slot + parity_base;
    const SlotMeta mt = p.slotMeta[sl];
    if (!warm_won && mt.timestep == tstep && mt.N == N && mt.a > 0) {   // uniform over the cluster
      const int a = mt.a;
      const int nv = mt.lsq ? a + 1 : a;
      const float* Vs = p.slotV32 + (size_t)sl * (p.max_a + 1) * p.slot_ld + base;
      block_partials_f32x<NT>(nv, [&](int i) {
        const float* vi = Vs + (size_t)i * p.slot_ld;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int l = tid + k * NT;
          if (l < SL) s = fmaf(vi[l], r[k], s);
        }
        return s;
      }, red32);
      cluster_sum(nv, true, no_tail);
      if (warp == 0) {
        __syncwarp();
        const double* rot = p.slotRot + (size_t)sl * 3 * p.max_a;
        solve_projected_warp(hb, a, mt.nrot, p.slotR + (size_t)sl * (p.max_a + 1) * p.max_a,
                             p.max_a + 1, rot, rot + 2 * p.max_a, lane);
        __syncwarp();
        for (int i = lane; i < a; i += 32) red32[i] = (float)hb[i];   // alpha in FP32, converted once
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int l = tid + k * NT;
        if (l < SL) {
          float xv = 0.f;
          for (int i = 0; i < a; ++i) xv = fmaf(red32[i], Vs[(size_t)i * p.slot_ld + l], xv);
          const dd xn = dd_add_f(dd{xh[l], xl[l]}, xv);
          xh[l] = xn.hi;
          xl[l] = xn.lo;
        }
      }
      r_current = false;
      proj_flops += (unsigned long long)(2 * nv + 2 * a) * (unsigned long long)N;
    }
  }
  if (p.x0_mode == X0_PROJECT) {
    const int sl = d.slot + parity_base;
    const SlotMeta mt = p.slotMeta[sl];
    if (mt.timestep == tstep && mt.N == N && mt.a > 0) {
      const int a = mt.a;
      const int nv = mt.lsq ? a + 1 : a;
      const float* Vs = p.slotV32 + (size_t)sl * (p.max_a + 1) * p.slot_ld + base;
      if (p.cproj) {
        if (tid < nv) hb[tid] = (double)p.cproj[(size_t)sysi * p.cproj_ld + tid];
        __syncthreads();
      } else {
        float bv[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) bv[k] = bhi(tid + k * NT);
        block_partials_f32x<NT>(nv, [&](int i) {
          const float* vi = Vs + (size_t)i * p.slot_ld;
          float s = 0.f;
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int l = tid + k * NT;
            if (l < SL) s = fmaf(vi[l], bv[k], s);
          }
          return s;
        }, red32);
        cluster_sum(nv, true, no_tail);
      }
      if (warp == 0) {
        __syncwarp();
        const double* rot = p.slotRot + (size_t)sl * 3 * p.max_a;
        solve_projected_warp(hb, a, mt.nrot, p.slotR + (size_t)sl * (p.max_a + 1) * p.max_a,
                             p.max_a + 1, rot, rot + 2 * p.max_a, lane);
        __syncwarp();
        for (int i = lane; i < a; i += 32) red32[i] = (float)hb[i];   // alpha in FP32, converted once
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int l = tid + k * NT;
        if (l < SL) {
          float xv = 0.f;
          for (int i = 0; i < a; ++i) xv = fmaf(red32[i], Vs[(size_t)i * p.slot_ld + l], xv);
          xh[l] = xv;
          xl[l] = 0.f;
        }
      }
      proj_flops = (unsigned long long)(2 * nv + 2 * a) * (unsigned long long)N;
    }
  }
  cluster.sync();                                 // x slices visible cluster-wide
  if (p.x0_mode == X0_ZERO) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) r[k] = bhi(tid + k * NT);
  } else if (!r_current) {
    residual();
  }
  block_partials_f32x<NT>(2, [&](int i) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const float v = (i == 0) ? bhi(tid + k * NT) : r[k];
      s = fmaf(v, v, s);
    }
    return s;
  }, red32);
  cluster_sum(2, true, no_tail);
  const double bnorm = sqrt(hb[0]);
  double beta = sqrt(hb[1]);
  int steps = 0, status = KP_NOT_CONVERGED, outer = 0;
  if (bnorm == 0.0) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) xh[tid + k * NT] = xl[tid + k * NT] = 0.f;
    beta = 0.0;
    status = KP_OK;
  }
  float w[EPT];
  while (status == KP_NOT_CONVERGED) {
    if (beta <= p.tol * bnorm) { status = KP_OK; break; }
    if (!isfinite(beta)) { status = KP_BREAKDOWN; break; }
    if (steps >= p.maxit || outer >= 64) break;
    const bool first = (outer == 0);
    const double target = (capture && first) ? p.tol * bnorm : fmax(kEta * beta, kInnerFloor * p.tol * bnorm);
    {
      const float ib = 1.f / (float)beta;
      float* v0 = vloc(0);
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int l = tid + k * NT;
        const float v = r[k] * ib;
        v0[l] = v;
        if (capture && first && l < SL) {
          capV[base + l] = v;
          if (p.capVb) p.capVb[(size_t)cidx * kVbRows * p.capVb_ld + base + l] = __float2bfloat16_rn(v);
        }
      }
      if (tid == 0) gv[0] = beta;
    }
    int kdone = 0, brk = 0;
    auto givens_step = [&](int j, double hn2) {
      const double ihn = hn2 > 0.0 ? rsqrt(hn2) : 0.0;
      const double hn = hn2 * ihn;
      const int b = !(hn2 > 1e-14 * sc[2]);      // hn <= 1e-7 ||w_0||: breakdown
      Hr[j + j * ld] += cd;                       // H_A = H_(A - cd I) + cd I
      Hr[(j + 1) + j * ld] = hn;
      if (capture && first && j < p.cap_a && rank == 0) {
        for (int i = 0; i <= j + 1; ++i) capH[i + j * (p.cap_a + 1)] = Hr[i + j * ld];
      }
      for (int i = 0; i < j; ++i) {
        const double t1 = Hr[i + j * ld], t2 = Hr[(i + 1) + j * ld];
        Hr[i + j * ld] = cs[i] * t1 + sn[i] * t2;
        Hr[(i + 1) + j * ld] = -sn[i] * t1 + cs[i] * t2;
      }
      const double a0 = Hr[j + j * ld];
      const double rr = a0 * a0 + hn2;
      const double ir = rsqrt(rr);
      const double c = a0 * ir, s = hn * ir;
      cs[j] = c;
      sn[j] = s;
      Hr[j + j * ld] = rr * ir;
      rinv[j] = ir;
      Hr[(j + 1) + j * ld] = 0.0;
      gv[j + 1] = -s * gv[j];
      gv[j] = c * gv[j];
      const double res = fabs(gv[j + 1]);
      sc[3] = ihn;
      fl[1] = b;
      // fixed basis dimension (as in the one-block mixed solver)
      const bool short_of_a = p.fixed_a && capture && first && j + 1 < p.cap_a;
      fl[2] = (res <= target && !short_of_a) || b || (steps >= p.maxit) || (j + 1 == m);
    };
    for (int j = 0; j < m; ++j) {
      cluster.sync();                             // v_j slices visible cluster-wide
      apply32(j, w);
      ++steps;
      const int nh = j + 1;
      auto dots = [&](int i) {
        float s = 0.f;
        if (i < nh) {
          const float* vi = vloc(i);
#pragma unroll
          for (int k = 0; k < EPT; ++k) s = fmaf(vi[tid + k * NT], w[k], s);
        } else {
#pragma unroll
          for (int k = 0; k < EPT; ++k) s = fmaf(w[k], w[k], s);
        }
        return s;
      };
      block_partials_f32x<NT>(nh + 1, dots, red32);
      cluster_sum(nh + 1, true, [&] {
        double sq = 0.0;
        for (int i = lane; i < nh; i += 32) { Hr[i + j * ld] = hb[i]; sq += hb[i] * hb[i]; }
        sq = warp_sum(sq);
        __syncwarp();
        if (lane == 0) {
          const double ww0 = hb[nh];
          sc[2] = ww0;
          const int pass2 = (p.reorth == 0) || (ww0 - sq < 0.5 * ww0);
          fl[0] = pass2;
          if (!pass2) givens_step(j, ww0 - sq);
        }
      });
      for (int i = 0; i < nh; ++i) {
        const float hi = hbf[i];
        const float* vi = vloc(i);
#pragma unroll
        for (int k = 0; k < EPT; ++k) w[k] = fmaf(-hi, vi[tid + k * NT], w[k]);
      }
      if (fl[0]) {
        block_partials_f32x<NT>(nh + 1, dots, red32);
        cluster_sum(nh + 1, true, [&] {
          double sq = 0.0;
          for (int i = lane; i < nh; i += 32) { Hr[i + j * ld] += hb[i]; sq += hb[i] * hb[i]; }
          sq = warp_sum(sq);
          __syncwarp();
          if (lane == 0) {
            const double ww1 = hb[nh];
            const int exact = sq > 0.25 * ww1;
            fl[3] = exact;
            if (!exact) givens_step(j, ww1 - sq);
          }
        });
        for (int i = 0; i < nh; ++i) {
          const float hi = hbf[i];
          const float* vi = vloc(i);
#pragma unroll
          for (int k = 0; k < EPT; ++k) w[k] = fmaf(-hi, vi[tid + k * NT], w[k]);
        }
        if (fl[3]) {
          block_partials_f32x<NT>(1, [&](int) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fmaf(w[k], w[k], s);
            return s;
          }, red32);
          cluster_sum(1, true, [&] {
            if (lane == 0) givens_step(j, hb[0]);
          });
        }
      }
      brk = fl[1];
      kdone = j + 1;
      if (!brk) {
        const float ih = (float)sc[3];
        float* vn = vloc(j + 1);
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int l = tid + k * NT;
          vn[l] = w[k] * ih;
          if (capture && first && j + 1 <= p.cap_a && l < SL) {
            capV[(size_t)(j + 1) * p.cap_ld + base + l] = w[k] * ih;
            if (p.capVb && j + 1 < kVbRows)
              p.capVb[((size_t)cidx * kVbRows + j + 1) * p.capVb_ld + base + l] = __float2bfloat16_rn(w[k] * ih);
          }
        }
      }
      if (fl[2]) break;
    }
    if (warp == 0) {
      double g0 = (lane < kdone) ? gv[lane] : 0.0;
      double g1 = (lane + 32 < kdone) ? gv[lane + 32] : 0.0;
      for (int i = kdone - 1; i >= 0; --i) {
        const double gi = __shfl_sync(kFull, i < 32 ? g0 : g1, i & 31);
        const double yi = gi * rinv[i];
        if (lane == 0) {
          yv[i] = yi;
          red32[i] = (float)yi;                     // y in FP32 for the update, converted once
        }
        if (lane < i) g0 = fma(-Hr[lane + i * ld], yi, g0);
        if (lane + 32 < i) g1 = fma(-Hr[(lane + 32) + i * ld], yi, g1);
      }
    }
    if (tid == 0 && rank == 0 && capture && first) {
      const int a = kdone < p.cap_a ? kdone : p.cap_a;
      const int hn = (a < kdone) || !brk;
      if (p.factor) {
        SlotMeta mt;
        double* rot = p.slotRot + (size_t)cidx * 3 * p.max_a;
        factor_hessenberg(capH, p.cap_a + 1, a, hn, p.slotR + (size_t)cidx * (p.max_a + 1) * p.max_a,
                          rot, rot + 2 * p.max_a, &mt.lsq, &mt.nrot);
        mt.a = a;
        mt.has_next = hn;
        mt.timestep = tstep;
        mt.N = N;
        mt.dense = mt.pad_ = 0;
        p.slotMeta[cidx] = mt;
      } else {
        p.capMeta[sysi].a = a;
        p.capMeta[sysi].has_next = hn;
        p.capMeta[sysi].N = N;
        p.capMeta[sysi].valid = 1;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int l = tid + k * NT;
      float dv = 0.f;
      for (int i = 0; i < kdone; ++i) dv = fmaf(red32[i], vloc(i)[l], dv);
      const dd xn = dd_add_f(dd{xh[l], xl[l]}, dv);
      xh[l] = xn.hi;
      xl[l] = xn.lo;
    }
    cluster.sync();                               // x slices visible cluster-wide
    residual();
    block_partials_f32x<NT>(1, [&](int) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < EPT; ++k) s = fmaf(r[k], r[k], s);
      return s;
    }, red32);
    cluster_sum(1, true, no_tail);
    beta = sqrt(hb[0]);
    ++outer;
  }
  if (capture && outer == 0 && tid == 0 && rank == 0) {
    if (p.factor) {
      SlotMeta mt;
      mt.a = 0; mt.has_next = 0; mt.timestep = tstep; mt.N = N; mt.lsq = 0; mt.nrot = 0;
      mt.dense = mt.pad_ = 0;
      p.slotMeta[cidx] = mt;
    } else {
      p.capMeta[sysi].a = 0;
      p.capMeta[sysi].has_next = 0;
      p.capMeta[sysi].N = N;
      p.capMeta[sysi].valid = 1;
    }
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int l = tid + k * NT;
    if (l < SL) {
      d.x[base + l] = dd_to_double(dd{xh[l], xl[l]});
      if (p.bnext)
        p.bnext[(size_t)sysi * p.bnext_ld + base + l] = __float2bfloat16_rn(xh[l]);
    }
  }
  if (tid == 0 && rank == 0) {
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
      const unsigned long long fl64 = (unsigned long long)(14 + outer * 13) * (unsigned long long)N;
      const unsigned long long fl32 = (gmres_flops(steps, m) - 14ull) * (unsigned long long)N;
      if (p.acc_kind == 0) {
        atomicAdd(&a->seed_iters, (unsigned long long)steps);
        atomicAdd(&a->seed_flops, fl64 + fl32);
      } else {
        atomicAdd(&a->tgt_iters, (unsigned long long)steps);
        atomicAdd(&a->tgt_flops, fl64);
        atomicAdd(&a->tgt_flops32, fl32);
        atomicMax(&a->tgt_max_iters, (unsigned int)steps);
        atomicMax(&a->max_res_bits, (unsigned long long)__double_as_longlong(rel));
        if (proj_flops) atomicAdd(&a->proj_flops, proj_flops);
      }
      if (status != KP_OK) atomicAdd(&a->not_converged, 1u);
    }
  }
  cluster.sync();                                 // no CTA leaves while others read its memory
}

template <int EPT, int NT, int CS, int MINB>
cudaError_t launch_c(const GmresParams& p, size_t smem, cudaStream_t st) {
  auto k = gmres_cluster_kernel<EPT, NT, CS, MINB>;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess && CS > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(p.nsys * CS));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

size_t gmres_cluster_smem_bytes(int ept, int nt, int S, int m) {
  const int npad = ept * nt;
  const size_t doubles = (size_t)npad + (nt / 32) * kMaxV + kMaxV + 2 * kMaxV +
                         (size_t)(m + 1) * m + (m + 1) + 4 * m + 8;
  return doubles * sizeof(double) + 8 * sizeof(int) + kMaxV * sizeof(float) + (size_t)S * npad * sizeof(float);
}

cudaError_t launch_gmres_cluster(const GmresParams& p, int ept, int nt, int cs, int minb, size_t smem,
                                 cudaStream_t st) {
  if (ept != 8) return cudaErrorInvalidValue;
  if (nt == 128) {
    // 16-CTA clusters of 128 threads (1024 points per CTA): up to four
    // systems' CTAs per SM
    if (cs != 16) return cudaErrorInvalidValue;
    if (minb == 4) return launch_c<8, 128, 16, 4>(p, smem, st);
    if (minb == 2) return launch_c<8, 128, 16, 2>(p, smem, st);
    return cudaErrorInvalidValue;
  }
  if (nt != 256) return cudaErrorInvalidValue;
  if (minb == 2) {
    if (cs == 8) return launch_c<8, 256, 8, 2>(p, smem, st);
    if (cs == 4) return launch_c<8, 256, 4, 2>(p, smem, st);
    if (cs == 2) return launch_c<8, 256, 2, 2>(p, smem, st);
  } else {
    if (cs == 8) return launch_c<8, 256, 8, 1>(p, smem, st);
    if (cs == 4) return launch_c<8, 256, 4, 1>(p, smem, st);
    if (cs == 2) return launch_c<8, 256, 2, 1>(p, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace kp
