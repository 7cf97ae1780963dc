// kp_gmres_mixed.cu -- mixed-precision solver for the five-point systems of
// Sec. 2.3: iterative refinement around an FP32 restarted GMRES.
//
// On GB300 an SM retires about 2 FP64 FMAs per clock against 128 FP32 FMAs,
// so the Krylov work (stencil, Gram-Schmidt updates, normalisation) runs in
// FP32 on FP32 vectors held in shared memory, and the refinement's
// high-precision arithmetic -- the solution x, the operator coefficients and
// the true residual r = b - A x -- runs in double-float (kp_dd.cuh: a pair of
// floats, about 48 bits) on the FP32 pipe as well, with FP64 inputs split by
// integer operations and the solution written back as FP64.  The residual's
// error is a few units of 2^-44 times ||b||, far below every tolerance the
// solver is asked for (>= 1e-12):
//   * inner products of FP32 vectors are summed in FP32 within a warp (its
//     few hundred products) and across warps, then held as FP64 numbers: the
//     Gram-Schmidt coefficients of both CGS passes, all norms and the residual
//     norms;
//   * the Hessenberg matrix, Givens rotations and least-squares solve are FP64.
// Outer loop: r = b - A x (double-float); inner GMRES(m) on A d = r in FP32
// until the residual estimate drops by eta = 1e-5 (FP32 cannot resolve much
// more) or to half the outer target (kInnerFloor); x += d.  The outer loop
// stops on the true residual, so every returned solve meets
// ||b - A x|| <= tol ||b||.
//
// The operator is applied from q_x = f_x/(2h) - e (m~_E - m~_W) and q_y per
// point (two numbers instead of four coefficients, which keeps the 4096-point
// instance within its registers):
//   A x = cd x_p - c (x_E + x_W + x_N + x_S) + q_x (x_E - x_W) + q_y (x_N - x_S)
// with out-of-grid neighbours zero -- algebraically the coefficients of the
// listing after Eq. 11.  The Arnoldi process runs on A - cd I (same Krylov
// space, H_A = H + cd I), which avoids the cancellation of the large
// diagonal in Gram-Schmidt -- in FP32 it would cost a digit per step.
#include "kp_dd.cuh"
#include "kp_internal.cuh"

namespace kp {
namespace {

struct SmemM {
  float* V;      // [S][npad] FP32 Krylov vectors
  float* xh;     // [npad] solution, double-float hi
  float* xl;     // [npad] and lo parts
  double* red;   // [NWARPS][kMaxV]
  double* hb;    // [kMaxV]
  double* Hr;    // [(m+1) * m]
  double* g;     // [m+1]
  double* cs;    // [m]
  double* sn;    // [m]
  double* y;     // [m]
  double* rinv;  // [m]
  double* sc;    // [8]
  int* fl;       // [8]
};

__device__ __forceinline__ SmemM carve_m(double* base, int npad, int nwarps, int m, int S) {
  SmemM s;
  s.xh = reinterpret_cast<float*>(base);
  s.xl = s.xh + npad;
  s.red = base + npad;
  s.hb = s.red + nwarps * kMaxV;
  s.Hr = s.hb + kMaxV;
  s.g = s.Hr + (m + 1) * m;
  s.cs = s.g + (m + 1);
  s.sn = s.cs + m;
  s.y = s.sn + m;
  s.rinv = s.y + m;
  s.sc = s.rinv + m;
  s.fl = reinterpret_cast<int*>(s.sc + 8);
  s.V = reinterpret_cast<float*>(s.fl + 8);
  (void)S;
  return s;
}

template <int EPT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) gmres_mixed_kernel(const GmresParams p) {
  constexpr int NWARPS = NT / 32;
  extern __shared__ __align__(16) double smem_raw[];
  const int npad = EPT * NT;
  const int m = p.m;
  const int ld = m + 1;
  SmemM sm = carve_m(smem_raw, npad, NWARPS, m, p.S);
  float* red32 = reinterpret_cast<float*>(sm.red);   // FP32 per-warp partials
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* spill = p.spill32 ? p.spill32 + (size_t)blockIdx.x * (m + 1 - p.S) * npad : nullptr;
  auto slot = [&](int i) -> float* {
    return i < p.S ? sm.V + (size_t)i * npad : spill + (size_t)(i - p.S) * npad;
  };
  int tstep = 0;
  if (p.step) {
    tstep = *p.step + p.step_offset;
    if (tstep >= *p.step_end) return;
  }
  const int parity_base = slot_set_base(p, tstep);
  const double bsc = p.b_scale;
  const double kEta = p.inner_eta > 0.0 ? p.inner_eta : 1e-5;   // inner residual reduction per outer step

  for (int sysi = blockIdx.x; sysi < p.nsys; sysi += gridDim.x) {
    const SysDesc d = p.sys[sysi];
    const int H = d.H, W = d.W, N = H * W;
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
    const bool drift = d.fx != nullptr || d.fy != nullptr;
    const bool capture = p.capV32 != nullptr;
    const int cidx = p.factor ? parity_base + sysi : sysi;
    float* capV = capture ? p.capV32 + (size_t)cidx * (p.cap_a + 1) * p.cap_ld : nullptr;
    double* capH = capture ? p.capH + (size_t)cidx * (p.cap_a + 1) * p.cap_a : nullptr;

    // q_x, q_y per point (FP32 copies for the Krylov operator), the
    // double-float E and N coefficients cE = q_x - c, cN = q_y - c for the
    // residual (W and S follow: cW = -2c - cE, cS = -2c - cN), and neighbour
    // masks; in the judge mode (a given guess) the warm start's residual norm
    // comes out of the same loads: sw = sum of r_warm^2 over this thread's points
    const bool judge = p.x0_mode == X0_GUESS_PROJECT;
    const dd ccd = dd_from_double(cc), eed = dd_from_double(ee), cdd = dd_from_double(cd);
    const dd i2hd = dd_from_double(i2h), c2d = dd_from_double(2.0 * cc);
    dd cE[EPT], cN[EPT];
    float qxf[EPT], qyf[EPT];
    unsigned msk[EPT];                          // bit0 E, bit1 W, bit2 N, bit3 S present
    float sw = 0.f;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      dd qx = {0.f, 0.f}, qy = {0.f, 0.f};
      msk[k] = 0;
      if (pp < N) {
        const int i = pp / H, j = pp - i * H;
        msk[k] = (i + 1 < W ? 1u : 0u) | (i > 0 ? 2u : 0u) | (j + 1 < H ? 4u : 0u) | (j > 0 ? 8u : 0u);
        const dd mE = dd_from_double((msk[k] & 1u) ? d.mt[pp + H] : 0.0);
        const dd mW = dd_from_double((msk[k] & 2u) ? d.mt[pp - H] : 0.0);
        const dd mN = dd_from_double((msk[k] & 4u) ? d.mt[pp + 1] : 0.0);
        const dd mS = dd_from_double((msk[k] & 8u) ? d.mt[pp - 1] : 0.0);
        qx = dd_mul(eed, dd_sub(mW, mE));
        qy = dd_mul(eed, dd_sub(mS, mN));
        if (drift) {
          if (d.fx) qx = dd_add(qx, dd_mul(dd_from_double(d.fx[pp]), i2hd));
          if (d.fy) qy = dd_add(qy, dd_mul(dd_from_double(d.fy[pp]), i2hd));
        }
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
    // r = b - A x in double-float with the masked neighbours (A x = cd x +
    // cE (xE - xW) - 2c xW + cN (xN - xS) - 2c xS); out = its hi part, which
    // is all the FP32 Krylov and the norms need
    auto residual_of = [&](float (&out)[EPT]) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        out[k] = 0.f;
        if (pp < N) {
          const dd z = {0.f, 0.f};
          const dd xE = (msk[k] & 1u) ? dd{sm.xh[pp + H], sm.xl[pp + H]} : z;
          const dd xW = (msk[k] & 2u) ? dd{sm.xh[pp - H], sm.xl[pp - H]} : z;
          const dd xN = (msk[k] & 4u) ? dd{sm.xh[pp + 1], sm.xl[pp + 1]} : z;
          const dd xS = (msk[k] & 8u) ? dd{sm.xh[pp - 1], sm.xl[pp - 1]} : z;
          dd t = dd_sub(dd_from_double(d.b[pp]), dd_mul(cdd, dd{sm.xh[pp], sm.xl[pp]}));
          t = dd_sub(t, dd_mul(cE[k], dd_sub(xE, xW)));
          t = dd_sub(t, dd_mul(cN[k], dd_sub(xN, xS)));
          t = dd_add(t, dd_mul(c2d, dd_add(xW, xS)));
          out[k] = t.hi;
        }
      }
    };
    auto apply32 = [&](const float* v, float (&out)[EPT]) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        out[k] = 0.f;
        if (pp < N) {
          const float xE = (msk[k] & 1u) ? v[pp + H] : 0.f;
          const float xW = (msk[k] & 2u) ? v[pp - H] : 0.f;
          const float xN = (msk[k] & 4u) ? v[pp + 1] : 0.f;
          const float xS = (msk[k] & 8u) ? v[pp - 1] : 0.f;
          out[k] = -ccf * (xE + xW + xN + xS) + qxf[k] * (xE - xW) + qyf[k] * (xN - xS);
        }
      }
    };
    auto bhi = [&](int pp) { return (pp < N) ? dd_from_double(d.b[pp]).hi : 0.f; };
    // x from an FP64 field (or zero), split into double-float
    auto load_x = [&](const double* src) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        const dd v = (src && pp < N) ? dd_from_double(src[pp]) : dd{0.f, 0.f};
        sm.xh[pp] = v.hi;
        sm.xl[pp] = v.lo;
      }
    };

    // initial guess
    if (p.gdelta && (p.x0_mode == X0_READ || judge)) {
      // the learned guess x_init = m~ + dt rho net, from the network's FP32
      // output, in double-float
      const float sg = (float)(p.grho[sysi] / p.gdiv);
      const float* dl = p.gdelta + (size_t)sysi * p.gdelta_ld;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        const dd v = pp < N ? dd_add_f(dd_from_double(d.mt[pp]), sg * dl[pp]) : dd{0.f, 0.f};
        sm.xh[pp] = v.hi;
        sm.xl[pp] = v.lo;
      }
    } else {
      load_x(p.x0_mode == X0_READ || judge ? d.x : p.x0_mode == X0_WARM ? d.mt : nullptr);
    }
    unsigned long long proj_flops = 0;
    float r[EPT];
    auto residual = [&]() { residual_of(r); };
    bool r_current = false;                         // r already holds b - A x0
    if (judge) {
      // the judge of a given guess (the learned one): its true residual
      // against the warm start's (sw, from the set-up); a kept guess is
      // projected below, the warm start (the fallback) starts unprojected, as
      // in the warm mode
      __syncthreads();                              // x_init complete for the stencil
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
      if (warp == 0) {
        cross_warp_f32<NT>(red32, 2, sm.hb, lane);
        __syncwarp();
        if (lane == 0) sm.fl[5] = sm.hb[1] < sm.hb[0];
      }
      __syncthreads();
      if (sm.fl[5]) load_x(d.mt);                   // the warm start wins
      r_current = !sm.fl[5];
      proj_flops = 26ull * (unsigned long long)N;
      // Sec. 3, Phase 2 on the residual of the guess: r = b - A x_init
      // (double-float), c = V^T r (FP32 products and sums), alpha = H_a^{-1} c
      // (FP64), x0 = x_init + V alpha
      const int sl = d.slot + parity_base;
      const SlotMeta mt = p.slotMeta[sl];
      if (!sm.fl[5] && mt.timestep == tstep && mt.N == N && mt.a > 0) {   // uniform per block
        const int a = mt.a;
        const int nv = mt.lsq ? a + 1 : a;
        const float* V = p.slotV32 + (size_t)sl * (p.max_a + 1) * p.slot_ld;
        block_partials_f32x<NT>(nv, [&](int i) {
          const float* vi = V + (size_t)i * p.slot_ld;
          float s = 0.f;
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            if (pp < N) s = fmaf(vi[pp], r[k], s);
          }
          return s;
        }, red32);
        if (warp == 0) {
          cross_warp_f32<NT>(red32, nv, sm.hb, lane);
          __syncwarp();
          const double* rot = p.slotRot + (size_t)sl * 3 * p.max_a;
          solve_projected_warp(sm.hb, a, mt.nrot, p.slotR + (size_t)sl * (p.max_a + 1) * p.max_a,
                               p.max_a + 1, rot, rot + 2 * p.max_a, lane);
          __syncwarp();
          for (int i = lane; i < a; i += 32) red32[i] = (float)sm.hb[i];   // alpha in FP32, converted once
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          if (pp < N) {
            float xv = 0.f;
            for (int i = 0; i < a; ++i) xv = fmaf(red32[i], V[(size_t)i * p.slot_ld + pp], xv);
            const dd xn = dd_add_f(dd{sm.xh[pp], sm.xl[pp]}, xv);
            sm.xh[pp] = xn.hi;
            sm.xl[pp] = xn.lo;
          }
        }
        r_current = false;
        proj_flops += (unsigned long long)(2 * nv + 2 * a) * (unsigned long long)N;
      }
    }
    if (p.x0_mode == X0_PROJECT) {
      // Sec. 3, Phase 2 with the seed's FP32 basis: c = V^T b (FP32 products and sums),
      // alpha = H_a^{-1} c (FP64), x0 = V alpha
      const int sl = d.slot + parity_base;
      const SlotMeta mt = p.slotMeta[sl];
      if (mt.timestep == tstep && mt.N == N && mt.a > 0) {
        const int a = mt.a;
        const int nv = mt.lsq ? a + 1 : a;
        const float* V = p.slotV32 + (size_t)sl * (p.max_a + 1) * p.slot_ld;
        if (p.cproj) {
          // c computed beforehand (tensor-core projection GEMM)
          if (tid < nv) sm.hb[tid] = (double)p.cproj[(size_t)sysi * p.cproj_ld + tid];
          __syncthreads();
        } else {
          float bv[EPT];
#pragma unroll
          for (int k = 0; k < EPT; ++k) bv[k] = bhi(tid + k * NT);
          block_partials_f32x<NT>(nv, [&](int i) {
            const float* vi = V + (size_t)i * p.slot_ld;
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
              const int pp = tid + k * NT;
              if (pp < N) s = fmaf(vi[pp], bv[k], s);
            }
            return s;
          }, red32);
          if (warp == 0) cross_warp_f32<NT>(red32, nv, sm.hb, lane);
        }
        if (warp == 0) {
          __syncwarp();
          const double* rot = p.slotRot + (size_t)sl * 3 * p.max_a;
          solve_projected_warp(sm.hb, a, mt.nrot, p.slotR + (size_t)sl * (p.max_a + 1) * p.max_a,
                               p.max_a + 1, rot, rot + 2 * p.max_a, lane);
          __syncwarp();
          for (int i = lane; i < a; i += 32) red32[i] = (float)sm.hb[i];   // alpha in FP32, converted once
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          if (pp < N) {
            float xv = 0.f;
            for (int i = 0; i < a; ++i) xv = fmaf(red32[i], V[(size_t)i * p.slot_ld + pp], xv);
            sm.xh[pp] = xv;
            sm.xl[pp] = 0.f;
          }
        }
        proj_flops = (unsigned long long)(2 * nv + 2 * a) * (unsigned long long)N;
      }
    }
    if (p.x0_mode == X0_GALERKIN && p.gram) {
      // Sec. 3, Phase 2 without the seed-matrix shortcut: G alpha = V_a^T b
      // with G = V_a^T A_i V_a of this target's own operator, assembled from
      // the seed basis part G0 and this target's tensor-core part (kp_gram.cu),
      // x0 = V_a alpha; c = V^T b from the projection GEMM
      const int sl = d.slot + parity_base;
      const SlotMeta mt = p.slotMeta[sl];
      const int a = mt.a, A = p.gram_a;
      if (mt.timestep == tstep && mt.N == N && a > 0 && a <= A && a * a <= (m + 1) * m && p.cproj) {
        const float* V = p.slotV32 + (size_t)sl * (p.max_a + 1) * p.slot_ld;
        const float* g0 = p.gram0 + (size_t)sl * A * A;
        const float* gi = p.gram + (size_t)sysi * A * A;
        double* G = sm.Hr;                          // a x a, column-major: G[l + k a] = v_l^T A v_k
        for (int e = tid; e < a * a; e += NT) {
          const int l = e % a, k = e / a;
          G[e] = (double)g0[l * A + k] + (double)gi[l * A + k];
        }
        if (tid < a) sm.hb[tid] = (double)p.cproj[(size_t)sysi * p.cproj_ld + tid];
        __syncthreads();
        if (warp == 0) {
          const bool ok = lu_solve_warp(G, a, sm.hb, lane);
          for (int i = lane; i < a; i += 32) red32[i] = (float)sm.hb[i];
          if (lane == 0) sm.fl[5] = ok;
        }
        __syncthreads();
        if (sm.fl[5]) {
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            if (pp < N) {
              float xv = 0.f;
              for (int i = 0; i < a; ++i) xv = fmaf(red32[i], V[(size_t)i * p.slot_ld + pp], xv);
              sm.xh[pp] = xv;
              sm.xl[pp] = 0.f;
            }
          }
        }
        proj_flops = (unsigned long long)(2 * a) * (unsigned long long)N;
      }
    }
    __syncthreads();
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
    if (warp == 0) {
      cross_warp_f32<NT>(red32, 2, sm.hb, lane);
      __syncwarp();
      if (lane == 0) {
        sm.sc[0] = sqrt(sm.hb[0]);
        sm.sc[1] = sqrt(sm.hb[1]);
      }
    }
    __syncthreads();
    const double bnorm = sm.sc[0];
    double beta = sm.sc[1];
    int steps = 0, status = KP_NOT_CONVERGED, outer = 0, restarts = 0;
    if (bnorm == 0.0) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) sm.xh[tid + k * NT] = sm.xl[tid + k * NT] = 0.f;
      beta = 0.0;
      status = KP_OK;
    }
    float w[EPT];
    while (status == KP_NOT_CONVERGED) {
      if (beta <= p.tol * bnorm) { status = KP_OK; break; }
      if (!isfinite(beta)) { status = KP_BREAKDOWN; break; }
      if (steps >= p.maxit || outer >= 64) break;
      const bool first = (outer == 0);
      // the seed's captured cycle runs to the seed tolerance, so its basis has
      // the dimension the FP64 method would keep (Sec. 3, Phase 1)
      const double target = (capture && first) ? p.tol * bnorm : fmax(kEta * beta, kInnerFloor * p.tol * bnorm);
      // ---- inner FP32 GMRES(m) on A d = r, from d = 0
      {
        const float ib = 1.f / (float)beta;
        float* v0 = slot(0);
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          const float v = r[k] * ib;
          v0[pp] = v;
          if (capture && first && pp < N) {
            capV[pp] = v;
            if (p.capVb) p.capVb[(size_t)cidx * kVbRows * p.capVb_ld + pp] = __float2bfloat16_rn(v);
          }
        }
        if (tid == 0) sm.g[0] = beta;
      }
      int kdone = 0, brk = 0;
      auto givens_step = [&](int j, double hn2) {
        const double ihn = hn2 > 0.0 ? rsqrt(hn2) : 0.0;
        const double hn = hn2 * ihn;
        const int b = !(hn > 1e-7 * sqrt(sm.sc[2]));      // FP32 vectors: breakdown at FP32 level
        sm.Hr[j + j * ld] += cd;                 // H_A = H_(A - cd I) + cd I
        sm.Hr[(j + 1) + j * ld] = hn;
        if (capture && first && j < p.cap_a) {
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
        // fixed basis dimension: the seed's captured cycle reaches cap_a steps
        // before the residual test may end it
        const bool short_of_a = p.fixed_a && capture && first && j + 1 < p.cap_a;
        sm.fl[2] = (res <= target && !short_of_a) || b || (steps >= p.maxit) || (j + 1 == m);
      };
      for (int j = 0; j < m; ++j) {
        __syncthreads();
        apply32(slot(j), w);
        ++steps;
        const int nh = j + 1;
        auto dots = [&](int i) {
          float s = 0.f;
          if (i < nh) {
            const float* vi = slot(i);
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fmaf(vi[tid + k * NT], w[k], s);
          } else {
#pragma unroll
            for (int k = 0; k < EPT; ++k) s = fmaf(w[k], w[k], s);
          }
          return s;
        };
        block_partials_f32x<NT>(nh + 1, dots, red32);
        if (warp == 0) {
          cross_warp_f32<NT>(red32, nh + 1, sm.hb, lane);
          __syncwarp();
          double sq = 0.0;
          for (int i = lane; i < nh; i += 32) {
            const double s = sm.hb[i];
            sm.Hr[i + j * ld] = s;
            sq += s * s;
          }
          sq = warp_sum(sq);
          if (lane == 0) {
            const double ww0 = sm.hb[nh];
            sm.sc[2] = ww0;
            const int pass2 = (p.reorth == 0) || (ww0 - sq < 0.5 * ww0);
            sm.fl[0] = pass2;
            if (!pass2) givens_step(j, ww0 - sq);
          }
        }
        __syncthreads();
        for (int i = 0; i < nh; ++i) {
          const float hi = (float)sm.hb[i];
          const float* vi = slot(i);
#pragma unroll
          for (int k = 0; k < EPT; ++k) w[k] = fmaf(-hi, vi[tid + k * NT], w[k]);
        }
        if (sm.fl[0]) {
          block_partials_f32x<NT>(nh + 1, dots, red32);
          if (warp == 0) {
            cross_warp_f32<NT>(red32, nh + 1, sm.hb, lane);
            __syncwarp();
            double sq = 0.0;
            for (int i = lane; i < nh; i += 32) {
              const double s = sm.hb[i];
              sm.Hr[i + j * ld] += s;
              sq += s * s;
            }
            sq = warp_sum(sq);
            if (lane == 0) {
              const double ww1 = sm.hb[nh];
              const int exact = sq > 0.25 * ww1;
              sm.fl[3] = exact;
              if (!exact) givens_step(j, ww1 - sq);
            }
          }
          __syncthreads();
          for (int i = 0; i < nh; ++i) {
            const float hi = (float)sm.hb[i];
            const float* vi = slot(i);
#pragma unroll
            for (int k = 0; k < EPT; ++k) w[k] = fmaf(-hi, vi[tid + k * NT], w[k]);
          }
          if (sm.fl[3]) {
            block_partials_f32x<NT>(1, [&](int) {
              float s = 0.f;
#pragma unroll
              for (int k = 0; k < EPT; ++k) s = fmaf(w[k], w[k], s);
              return s;
            }, red32);
            if (warp == 0) {
              cross_warp_f32<NT>(red32, 1, sm.sc + 5, lane);
              __syncwarp();
              if (lane == 0) givens_step(j, sm.sc[5]);
            }
            __syncthreads();
          }
        }
        brk = sm.fl[1];
        kdone = j + 1;
        if (!brk) {
          const float ih = (float)sm.sc[3];
          float* vn = slot(j + 1);
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            vn[pp] = w[k] * ih;
            if (capture && first && j + 1 <= p.cap_a && pp < N) {
              capV[(size_t)(j + 1) * p.cap_ld + pp] = w[k] * ih;
              if (p.capVb && j + 1 < kVbRows)
                p.capVb[((size_t)cidx * kVbRows + j + 1) * p.capVb_ld + pp] = __float2bfloat16_rn(w[k] * ih);
            }
          }
        }
        if (sm.fl[2]) break;
      }
      if (warp == 0) {
        double g0 = (lane < kdone) ? sm.g[lane] : 0.0;
        double g1 = (lane + 32 < kdone) ? sm.g[lane + 32] : 0.0;
        for (int i = kdone - 1; i >= 0; --i) {
          const double gi = __shfl_sync(kFull, i < 32 ? g0 : g1, i & 31);
          const double yi = gi * sm.rinv[i];
          if (lane == 0) {
            sm.y[i] = yi;
            red32[i] = (float)yi;                   // y in FP32 for the update, converted once
          }
          if (lane < i) g0 = fma(-sm.Hr[lane + i * ld], yi, g0);
          if (lane + 32 < i) g1 = fma(-sm.Hr[(lane + 32) + i * ld], yi, g1);
        }
      }
      if (tid == 0 && capture && first) {
        const int a = kdone < p.cap_a ? kdone : p.cap_a;
        const int hn = (a < kdone) || !brk;
        if (p.factor) {
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
      __syncthreads();
      // d = V y in FP32, x += d in double-float
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        float dv = 0.f;
        for (int i = 0; i < kdone; ++i) dv = fmaf(red32[i], slot(i)[pp], dv);
        const dd xn = dd_add_f(dd{sm.xh[pp], sm.xl[pp]}, dv);
        sm.xh[pp] = xn.hi;
        sm.xl[pp] = xn.lo;
      }
      __syncthreads();
      residual();                                 // the true residual (double-float)
      block_partials_f32x<NT>(1, [&](int) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < EPT; ++k) s = fmaf(r[k], r[k], s);
        return s;
      }, red32);
      if (warp == 0) {
        cross_warp_f32<NT>(red32, 1, sm.hb, lane);
        __syncwarp();
        if (lane == 0) sm.sc[1] = sqrt(sm.hb[0]);
      }
      __syncthreads();
      beta = sm.sc[1];
      ++outer;
      ++restarts;
    }
    if (capture && outer == 0 && tid == 0) {
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
      const int pp = tid + k * NT;
      if (pp < N) {
        d.x[pp] = dd_to_double(dd{sm.xh[pp], sm.xl[pp]});
        if (p.bnext) p.bnext[(size_t)sysi * p.bnext_ld + pp] = __float2bfloat16_rn(sm.xh[pp]);
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
        // high-precision flops of the refinement (residuals, x update: in
        // double-float); FP32 Krylov work is counted separately
        const unsigned long long fl = (unsigned long long)(14 + restarts * 13) * (unsigned long long)N;
        const unsigned long long fl32 = (gmres_flops(steps, m) - 14ull) * (unsigned long long)N;
        if (p.acc_kind == 0) {
          atomicAdd(&a->seed_iters, (unsigned long long)steps);
          atomicAdd(&a->seed_flops, fl + fl32);
        } else {
          atomicAdd(&a->tgt_iters, (unsigned long long)steps);
          atomicAdd(&a->tgt_flops, fl);
          atomicAdd(&a->tgt_flops32, fl32);
          atomicMax(&a->tgt_max_iters, (unsigned int)steps);
          atomicMax(&a->max_res_bits, (unsigned long long)__double_as_longlong(rel));
          if (proj_flops) atomicAdd(&a->proj_flops, proj_flops);
        }
        if (status != KP_OK) atomicAdd(&a->not_converged, 1u);
      }
    }
    __syncthreads();
  }
}

template <typename K>
cudaError_t allow_max_smem_m(K k, size_t smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <int EPT, int NT, int MINB>
cudaError_t launch_m(const GmresParams& p, size_t smem, cudaStream_t st) {
  auto k = gmres_mixed_kernel<EPT, NT, MINB>;
  cudaError_t e = allow_max_smem_m(k, smem);
  if (e != cudaSuccess) return e;
  k<<<p.nsys, NT, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t gmres_mixed_smem_bytes(int ept, int nt, int S, int m) {
  const int npad = ept * nt;
  const size_t doubles = (size_t)npad + (nt / 32) * kMaxV + kMaxV + (size_t)(m + 1) * m +
                         (m + 1) + 4 * m + 8;
  return doubles * sizeof(double) + 8 * sizeof(int) + (size_t)S * npad * sizeof(float);
}

cudaError_t launch_gmres_mixed(const GmresParams& p, int ept, int nt, size_t smem,
                               cudaStream_t st) {
  if (ept == 4 && nt == 256) return launch_m<4, 256, 2>(p, smem, st);
  if (ept == 8 && nt == 128) return launch_m<8, 128, 2>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_m<8, 512, 1>(p, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
